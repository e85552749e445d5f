// kernels_generic.cu -- initial state, the general checkerboard half-sweep
// (any dims, spin value and model; two launches per sweep, one per colour,
// the kernel boundary being the device-wide barrier as in §III.A steps 6-7),
// the stand-alone measurement kernel and the planar <-> linear conversions.
// Spins use the checkerboard-planar int8 layout described in Geom.
#include <cmath>

#include <algorithm>

#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;

LAT_D int wrapc(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

LAT_D uint64_t addr(const Geom &g, int x, int y, int z)
{
    return planar_index(g, wrapc(x, g.L), wrapc(y, g.L), wrapc(z, g.L));
}

// §III.A step 1 / §III.B step 1: initial configuration, one Philox call per
// four consecutive (linear, x-fastest) sites with counter (i >> 2, 0, 0, 2).
__global__ void k_init(Geom g, int init, uint32_t thr_c)
{
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t i0 = q << 2;
    if (i0 >= g.N) return;
    const U4 u = philox(U4{(uint32_t)q, 0u, 0u, 2u}, g.key0, g.key1);
    for (int k = 0; k < 4 && i0 + k < g.N; ++k) {
        const uint64_t i = i0 + k;
        const uint32_t w = word_of(u, k);
        int st;
        if (init == LAT_INIT_COLD) {
            st = g.model == LAT_POTTS ? 0 : g.two_S;
        } else if (init == LAT_INIT_RANDOM) {
            if (g.two_S == 1) st = (w < 0x80000000u) == (g.model != LAT_POTTS) ? 1 : 0;   // Potts: state 0 <-> up
            else st = (int)(((uint64_t)w * (uint64_t)(g.two_S + 1)) >> 32);
        } else {
            st = (w < thr_c) ? 1 : 0;
        }
        const int x = (int)(i % (uint64_t)g.L);
        const int y = (int)((i / (uint64_t)g.L) % (uint64_t)g.L);
        const int z = (int)(i / ((uint64_t)g.L * (uint64_t)g.L));
        g.s[0][planar_index(g, x, y, z)] = (int8_t)(g.model == LAT_POTTS ? st : spin_of_state(g.two_S, st));
    }
}

// Partial per-sweep counters of one thread.
struct Part {
    long long bond = 0, mag = 0, up = 0, unfl = 0, acf = 0, fld = 0;
};

// Sweep the colour-`colour` sites of Philox group t = (row r, group m) of
// lattice g -- the same-colour sites j = m*2^sh .. m*2^sh + 2^sh - 1 of row
// r -- with the acceptance table in stab, and accumulate the colour-1
// counters into pt.
LAT_D void half_sweep_group(const Geom &g, const TabEntry *stab, int colour, unsigned long long sweep,
                            uint64_t t, Part &pt)
{
    const int8_t *src = g.s[sweep & 1];
    int8_t *dst = g.s[(sweep + 1) & 1];
    if (colour == 1) src = dst;
    const bool measure = (colour == 1);
    const uint32_t r = (uint32_t)t / g.G, m = (uint32_t)t - r * g.G;   // rows * G < 2^31
    const int L = g.L;
    const int y = (int)(r % (uint32_t)L), z = (int)(r / (uint32_t)L);
    const int p = (colour + y + z) & 1;
    const uint32_t grp = r * g.G + m;
    const U4 u = philox(U4{grp, (uint32_t)sweep, (uint32_t)(sweep >> 32), (uint32_t)colour},
                        g.key0, g.key1);
    const int per = 1 << g.sh;
    const int half = L >> 1;
    uint8_t *fl_c = g.flags ? g.flags + ((uint64_t)colour * g.rows + r) * g.G + m : nullptr;
    uint8_t *fl_o = g.flags ? g.flags + ((uint64_t)(1 - colour) * g.rows + r) * g.G + m : nullptr;
    uint32_t flips = 0;
    for (int q = 0; q < per; ++q) {
        const int j = (int)m * per + q;
        if (j >= half) break;
        const int x = 2 * j + p;
        const uint64_t i = addr(g, x, y, z);
        const uint64_t io = (uint64_t)(1 - colour) * g.plane + (uint64_t)r * g.half + (uint64_t)j;
        const int s_old = src[i];
        int n;
        int fo = 0;   // table half: the -h entries for a site with eta_i = -1
        if (g.cpl == nullptr) {
            n = src[addr(g, x - 1, y, z)] + src[addr(g, x + 1, y, z)] + src[addr(g, x, y - 1, z)] +
                src[addr(g, x, y + 1, z)];
            if (g.dims == 3) n += src[addr(g, x, y, z - 1)] + src[addr(g, x, y, z + 1)];
        } else {   // Eq. 1 disorder: sum of eps_ij * s_j, and the sign of B_i
            const uint32_t cb = g.cpl[i];
            auto sg = [&](int bit, int v) { return ((cb >> bit) & 1u) ? -v : v; };
            n = sg(0, src[addr(g, x - 1, y, z)]) + sg(1, src[addr(g, x + 1, y, z)]) +
                sg(2, src[addr(g, x, y - 1, z)]) + sg(3, src[addr(g, x, y + 1, z)]);
            if (g.dims == 3) n += sg(4, src[addr(g, x, y, z - 1)]) + sg(5, src[addr(g, x, y, z + 1)]);
            if ((cb >> 6) & 1u) fo = (2 * g.dsmax + 1) * g.nn;
        }
        const bool potts = g.model == LAT_POTTS;
        const int k_old = potts ? s_old : state_of_spin(g.two_S, s_old);
        int k_new;
        uint32_t u_acc;
        if (g.two_S == 1) {
            k_new = 1 - k_old;
            u_acc = word_of(u, j & 3);
        } else {
            const int w = 2 * (j & 1);
            u_acc = word_of(u, w);
            const uint32_t u_prop = word_of(u, w + 1);
            const int step = 1 + (int)(((uint64_t)u_prop * (uint64_t)g.two_S) >> 32);
            k_new = k_old + step;
            if (k_new > g.two_S) k_new -= g.two_S + 1;
        }
        const int s_new = potts ? k_new : spin_of_state(g.two_S, k_new);
        if (potts) {
            // Potts: dn = change in equal neighbours, df = change in the
            // state-0 indicator (labels are stored as the spin bytes)
            int nb[6];
            nb[0] = src[addr(g, x - 1, y, z)];
            nb[1] = src[addr(g, x + 1, y, z)];
            nb[2] = src[addr(g, x, y - 1, z)];
            nb[3] = src[addr(g, x, y + 1, z)];
            nb[4] = g.dims == 3 ? src[addr(g, x, y, z - 1)] : -1;
            nb[5] = g.dims == 3 ? src[addr(g, x, y, z + 1)] : -1;
            int dn = 0;
#pragma unroll
            for (int d = 0; d < 6; ++d) dn += (nb[d] == s_new) - (nb[d] == s_old);
            const int df = (s_new == 0) - (s_old == 0);
            const TabEntry e = stab[(df + 1) * g.nn + (dn + g.nmax)];
            int s_fin = s_old;
            if (e.always || u_acc < e.thr) s_fin = s_new;
            dst[i] = (int8_t)s_fin;
            if (colour == 0) dst[io] = src[io];
            if (measure) {
                int eq = 0;
#pragma unroll
                for (int d = 0; d < 6; ++d) eq += nb[d] == s_fin;
                pt.bond += eq;
                const int so = dst[io];
                pt.mag += (s_fin == 0) + (so == 0);
                pt.up += (s_fin != 0) + (so != 0);
                // overlap of labels: sites in their reference state
                if (g.ref != nullptr) pt.acf += (s_fin == g.ref[i]) + (so == g.ref[io]);
            }
            continue;
        }
        bool allowed = true;
        if (g.model == LAT_NE) {
            // §III.B: north (x, y-1) and east (x+1, y) must both be up.
            allowed = src[addr(g, x, y - 1, z)] == 1 && src[addr(g, x + 1, y, z)] == 1;
        }
        int s_fin = s_old;
        if (allowed) {
            const TabEntry e = stab[fo + (s_new - s_old + g.dsmax) * g.nn + (n + g.nmax)];
            if (e.always || u_acc < e.thr) {
                s_fin = s_new;
                if (s_new != s_old) flips |= 1u << q;
            }
        }
        dst[i] = (int8_t)s_fin;
        if (colour == 0) dst[io] = src[io];
        if (measure) {
            pt.bond += (long long)s_fin * n;
            const int so = dst[io];
            pt.mag += s_fin + so;
            pt.up += (s_fin > 0) + (so > 0);
            if (g.ref != nullptr) pt.acf += s_fin * g.ref[i] + so * g.ref[io];
            if (g.cpl != nullptr)
                pt.fld += (((g.cpl[i] >> 6) & 1u) ? -s_fin : s_fin) + (((g.cpl[io] >> 6) & 1u) ? -so : so);
        }
    }
    if (fl_c != nullptr) {
        const uint32_t f = *fl_c | flips;
        *fl_c = (uint8_t)f;
        if (measure) {
            const int valid = min(per, half - (int)m * per);
            const uint32_t vm = (1u << valid) - 1u;
            pt.unfl += valid - __popc(f & vm);
            pt.unfl += valid - __popc((uint32_t)*fl_o & vm);
        }
    }
}

LAT_D void flush_counters(const Geom &g, unsigned long long sweep, const Part &pt, long long *red)
{
    unsigned long long *slot = series_slot(g.ctrl, sweep);
    long long v;
    v = block_sum_ll(pt.bond, red);
    if (threadIdx.x == 0) add_counter(slot + 0, v);
    v = block_sum_ll(pt.mag, red);
    if (threadIdx.x == 0) add_counter(slot + 1, v);
    v = block_sum_ll(pt.up, red);
    if (threadIdx.x == 0) add_counter(slot + 2, v);
    v = block_sum_ll(pt.unfl, red);
    if (threadIdx.x == 0) add_counter(slot + 3, v);
    if (g.ref != nullptr) {
        v = block_sum_ll(pt.acf, red);
        if (threadIdx.x == 0) add_counter(acf_slot(g.ctrl, sweep), v);
    }
    if (g.cpl != nullptr) {
        v = block_sum_ll(pt.fld, red);
        if (threadIdx.x == 0) add_counter(fld_slot(g.ctrl, sweep), v);
    }
}

// One colour of one sweep (thread = Philox group).  Colour 0 reads buffer
// s[sweep & 1] and writes buffer s[(sweep+1) & 1] (new colour-0 values, and
// a copy of the colour-1 sites of the same j); colour 1 then works in place
// on s[(sweep+1) & 1] and accumulates the sweep's exact counters: bond
// (each bond has exactly one colour-1 end when L is even), magnetisation,
// up count and unflipped count over both colours of its j range.
__global__ void __launch_bounds__(kThreads) k_half_sweep(Geom g, int colour, int off)
{
    extern __shared__ TabEntry stab[];
    __shared__ long long red[kThreads / 32];
    for (int i = threadIdx.x; i < g.tab_n; i += blockDim.x) stab[i] = g.tab[i];
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    Part pt;
    if (t < (uint64_t)g.rows * g.G) half_sweep_group(g, stab, colour, sweep, t, pt);
    if (colour == 1) flush_counters(g, sweep, pt, red);
}

// Batched half-sweep: a persistent grid works through (lattice, chunk)
// items, a chunk being kThreads consecutive Philox groups of one lattice.
__global__ void __launch_bounds__(kThreads) k_batch_half_sweep(const Geom *geoms, const uint2 *items,
                                                              int n_items, unsigned *next_item,
                                                              int colour, int off)
{
    extern __shared__ TabEntry stab[];
    __shared__ long long red[kThreads / 32];
    __shared__ Geom sg;
    __shared__ int cur;
    for (;;) {
        if (threadIdx.x == 0) cur = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int it = cur;
        if (it >= n_items) break;
        const uint2 w = items[it];
        if (threadIdx.x < sizeof(Geom) / 4)
            reinterpret_cast<uint32_t *>(&sg)[threadIdx.x] =
                reinterpret_cast<const uint32_t *>(&geoms[w.x])[threadIdx.x];
        __syncthreads();
        for (int i = threadIdx.x; i < sg.tab_n; i += blockDim.x) stab[i] = sg.tab[i];
        const Geom g = sg;  // register copy: no aliasing with shared-memory stores
        __syncthreads();
        const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
        const uint64_t t = (uint64_t)w.y * kThreads + threadIdx.x;
        Part pt;
        if (t < (uint64_t)g.rows * g.G) half_sweep_group(g, stab, colour, sweep, t, pt);
        if (colour == 1) flush_counters(g, sweep, pt, red);
        __syncthreads();
    }
}

// After a batched sweep step: advance the sweep counter of every lattice of
// the step and clear the item counters for the next step.
__global__ void k_batch_advance(Ctrl *const *ctrls, int n, unsigned *counters, int n_counters,
                                unsigned long long k)
{
    dep_wait();   // the step's sweep kernels are done with the counters and sweep numbers
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ctrls[i]->sweep += k;
    if (i < n_counters) counters[i] = 0u;
    dep_launch();
}

// Counters of a configuration from their definitions (before the first
// sweep and after set_state): bond = sum over sites and directions of
// eps s_i s_{i+e_d}; mag; up; unflipped (from the persistence bytes); the
// field sum sum_i eta_i s_i.
__global__ void __launch_bounds__(kThreads) k_measure(Geom g, const int8_t *sp, unsigned long long *out)
{
    __shared__ long long red[kThreads / 32];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    long long bond = 0, mag = 0, up = 0, unfl = 0, fld = 0;
    if (i < g.N) {
        const int L = g.L;
        const int x = (int)(i % (uint64_t)L);
        const int y = (int)((i / (uint64_t)L) % (uint64_t)L);
        const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
        const uint64_t pi = planar_index(g, x, y, z);
        const int s = sp[pi];
        if (g.model == LAT_POTTS) {   // equal forward bonds, state-0 count, others
            int eq = (sp[addr(g, x + 1, y, z)] == s) + (sp[addr(g, x, y + 1, z)] == s);
            if (g.dims == 3) eq += sp[addr(g, x, y, z + 1)] == s;
            bond = eq;
            mag = s == 0;
            up = s != 0;
        } else {
            // forward bonds (+x, +y, +z), weighted by their coupling signs
            const uint32_t cb = g.cpl != nullptr ? g.cpl[pi] : 0u;
            auto sg = [&](int bit, int v) { return ((cb >> bit) & 1u) ? -v : v; };
            int nf = sg(1, sp[addr(g, x + 1, y, z)]) + sg(3, sp[addr(g, x, y + 1, z)]);
            if (g.dims == 3) nf += sg(5, sp[addr(g, x, y, z + 1)]);
            bond = (long long)s * nf;
            mag = s;
            up = s > 0;
            fld = ((cb >> 6) & 1u) ? -s : s;
        }
        if (g.flags != nullptr) {
            const int c = (x + y + z) & 1;
            const uint32_t r = (uint32_t)y + (uint32_t)L * (uint32_t)z;
            const uint32_t j = (uint32_t)x >> 1;
            const uint8_t f = g.flags[((uint64_t)c * g.rows + r) * g.G + (j >> g.sh)];
            unfl = ((f >> (j & ((1u << g.sh) - 1u))) & 1u) ? 0 : 1;
        }
    }
    long long v;
    v = block_sum_ll(bond, red);
    if (threadIdx.x == 0) add_counter(out + 0, v);
    v = block_sum_ll(mag, red);
    if (threadIdx.x == 0) add_counter(out + 1, v);
    v = block_sum_ll(up, red);
    if (threadIdx.x == 0) add_counter(out + 2, v);
    v = block_sum_ll(unfl, red);
    if (threadIdx.x == 0) add_counter(out + 3, v);
    v = block_sum_ll(fld, red);
    if (threadIdx.x == 0) add_counter(out + 4, v);
}

__global__ void k_to_linear(Geom g, const int8_t *planar, int8_t *linear)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const int L = g.L;
    const int x = (int)(i % (uint64_t)L);
    const int y = (int)((i / (uint64_t)L) % (uint64_t)L);
    const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
    linear[i] = planar[planar_index(g, x, y, z)];
}

__global__ void k_to_planar(Geom g, const int8_t *linear, int8_t *planar)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const int L = g.L;
    const int x = (int)(i % (uint64_t)L);
    const int y = (int)((i / (uint64_t)L) % (uint64_t)L);
    const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
    planar[planar_index(g, x, y, z)] = linear[i];
}

// Count the bytes of an uploaded spin array that are not allowed spin
// values (|v| > smax, or the wrong parity for half-integer S).
__global__ void __launch_bounds__(kThreads) k_count_bad(Geom g, const int8_t *s, unsigned long long *out)
{
    __shared__ long long red[kThreads / 32];
    const int smax = max_spin(g.two_S), odd = g.two_S & 1;
    long long bad = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < g.N; i += (uint64_t)gridDim.x * blockDim.x) {
        const int v = s[i];
        if (g.model == LAT_POTTS) bad += (v < 0) | (v > g.two_S);
        else bad += (v < -smax) | (v > smax) | (odd & ((v + g.two_S) & 1));
    }
    const long long t = block_sum_ll(bad, red);
    if (threadIdx.x == 0 && t != 0) atomicAdd(out, (unsigned long long)t);
}

__global__ void k_advance(Ctrl *ctrl, unsigned long long k) { ctrl->sweep += k; }

__global__ void k_set_ctrl(Ctrl *ctrl, unsigned long long sweep, unsigned long long *series,
                           unsigned long long base, unsigned long long cap, unsigned long long *acf,
                           unsigned long long *fld)
{
    ctrl->sweep = sweep;
    ctrl->series = series;
    ctrl->series_base = base;
    ctrl->series_cap = cap;
    ctrl->acf = acf;
    ctrl->fld = fld;
}

unsigned blocks_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_init(const Geom &g, int init, double c, cudaStream_t st)
{
    uint32_t thr_c = 0;
    if (init == LAT_INIT_EQUILIBRIUM) {
        // floor(c * 2^32), c in (0, 1): exact in double.
        thr_c = (uint32_t)floor(ldexp(c, 32));
    }
    k_init<<<blocks_for((g.N + 3) >> 2), kThreads, 0, st>>>(g, init, thr_c);
    return cudaGetLastError();
}

cudaError_t launch_half_sweep_generic(const Geom &g, int colour, int off, cudaStream_t st)
{
    const size_t smem = (size_t)g.tab_n * sizeof(TabEntry);
    k_half_sweep<<<blocks_for((uint64_t)g.rows * g.G), kThreads, smem, st>>>(g, colour, off);
    return cudaGetLastError();
}

cudaError_t launch_batch_generic(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                                 int colour, int off, int grid, int tab_max, cudaStream_t st)
{
    // The largest table (two_S <= 8, 3D) has 2465 entries, twice that with
    // per-site field signs.
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_batch_half_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * 2465 * sizeof(TabEntry)));
        attr = true;
    }
    const size_t smem = (size_t)tab_max * sizeof(TabEntry);
    k_batch_half_sweep<<<grid, kThreads, smem, st>>>(geoms, items, n_items, next_item, colour, off);
    return cudaGetLastError();
}

int batch_generic_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_half_sweep, kThreads, 2465 * sizeof(TabEntry));
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_advance(Ctrl *const *ctrls, int n, unsigned *counters, int n_counters,
                                 unsigned long long k, cudaStream_t st)
{
    const int m = n > n_counters ? n : n_counters;
    return launch_pdl(k_batch_advance, (unsigned)((m + kThreads - 1) / kThreads), kThreads, st, ctrls, n, counters,
                      n_counters, k);
}

cudaError_t launch_measure(const Geom &g, const int8_t *spins, unsigned long long *out5, cudaStream_t st)
{
    k_measure<<<blocks_for(g.N), kThreads, 0, st>>>(g, spins, out5);
    return cudaGetLastError();
}

cudaError_t launch_to_linear(const Geom &g, const int8_t *planar, int8_t *linear, cudaStream_t st)
{
    k_to_linear<<<blocks_for(g.N), kThreads, 0, st>>>(g, planar, linear);
    return cudaGetLastError();
}

cudaError_t launch_count_bad(const Geom &g, const int8_t *spins, unsigned long long *out, cudaStream_t st)
{
    const unsigned blocks = std::min<unsigned>(blocks_for(g.N), 4096u);
    k_count_bad<<<blocks, kThreads, 0, st>>>(g, spins, out);
    return cudaGetLastError();
}

cudaError_t launch_to_planar(const Geom &g, const int8_t *linear, int8_t *planar, cudaStream_t st)
{
    k_to_planar<<<blocks_for(g.N), kThreads, 0, st>>>(g, linear, planar);
    return cudaGetLastError();
}

cudaError_t launch_advance(Ctrl *ctrl, unsigned long long k, cudaStream_t st)
{
    k_advance<<<1, 1, 0, st>>>(ctrl, k);
    return cudaGetLastError();
}

cudaError_t launch_set_ctrl(Ctrl *ctrl, unsigned long long sweep, unsigned long long *series,
                            unsigned long long base, unsigned long long cap, unsigned long long *acf,
                            unsigned long long *fld, cudaStream_t st)
{
    k_set_ctrl<<<1, 1, 0, st>>>(ctrl, sweep, series, base, cap, acf, fld);
    return cudaGetLastError();
}

}  // namespace lat
