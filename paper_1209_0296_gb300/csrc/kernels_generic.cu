// kernels_generic.cu -- initial state, the general checkerboard half-sweep
// (any dims, spin value and model; two launches per sweep, one per colour,
// the kernel boundary being the device-wide barrier as in §III.A steps 6-7)
// and the stand-alone measurement kernel.
#include <cmath>

#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;

LAT_D uint64_t site_index(const Geom &g, int x, int y, int z)
{
    const int L = g.L;
    x = x < 0 ? x + L : (x >= L ? x - L : x);
    y = y < 0 ? y + L : (y >= L ? y - L : y);
    z = z < 0 ? z + L : (z >= L ? z - L : z);
    return (uint64_t)x + (uint64_t)L * ((uint64_t)y + (uint64_t)L * (uint64_t)z);
}

// §III.A step 1 / §III.B step 1: initial configuration, one Philox call per
// four consecutive sites with counter (i >> 2, 0, 0, 2).
__global__ void k_init(Geom g, int init, uint32_t thr_c)
{
    const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t i0 = q << 2;
    if (i0 >= g.N) return;
    U4 u = philox(U4{(uint32_t)q, 0u, 0u, 2u}, g.key0, g.key1);
    for (int k = 0; k < 4 && i0 + k < g.N; ++k) {
        const uint32_t w = word_of(u, k);
        int st;
        if (init == LAT_INIT_COLD) {
            st = g.two_S;
        } else if (init == LAT_INIT_RANDOM) {
            st = (g.two_S == 1) ? (w < 0x80000000u ? 1 : 0)
                                : (int)(((uint64_t)w * (uint64_t)(g.two_S + 1)) >> 32);
        } else {
            st = (w < thr_c) ? 1 : 0;
        }
        g.s[0][i0 + k] = (int8_t)spin_of_state(g.two_S, st);
    }
}

// One colour of one sweep.  Thread t handles Philox group (row r, group m):
// the same-colour sites j = m*2^sh .. m*2^sh + 2^sh - 1 of row r.
// Colour 0 reads buffer s[sweep & 1] and writes buffer s[(sweep+1) & 1]
// (new colour-0 values, and a copy of the colour-1 sites of the same
// columns); colour 1 then works in place on s[(sweep+1) & 1].  The colour-1
// launch also accumulates the sweep's exact counters: bond (each bond has
// exactly one colour-1 end when L is even), magnetisation, up count and
// unflipped count over both colours of its sites' columns.
__global__ void __launch_bounds__(kThreads) k_half_sweep(Geom g, int colour, int off)
{
    extern __shared__ TabEntry stab[];
    __shared__ long long red[kThreads / 32];
    for (int i = threadIdx.x; i < g.tab_n; i += blockDim.x) stab[i] = g.tab[i];
    __syncthreads();

    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const int8_t *src = g.s[sweep & 1];
    int8_t *dst = g.s[(sweep + 1) & 1];
    if (colour == 1) src = dst;
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)g.rows * g.G;
    const bool measure = (colour == 1);
    long long bond = 0, mag = 0, up = 0, unfl = 0;

    if (t < total) {
        const uint32_t r = (uint32_t)(t / g.G), m = (uint32_t)(t % g.G);
        const int L = g.L;
        const int y = (int)(r % (uint32_t)L), z = (int)(r / (uint32_t)L);
        const int p = (colour + y + z) & 1;
        const uint32_t grp = r * g.G + m;
        const U4 u = philox(U4{grp, (uint32_t)sweep, (uint32_t)(sweep >> 32), (uint32_t)colour},
                            g.key0, g.key1);
        const int per = 1 << g.sh;
        const int half = L >> 1;
        for (int q = 0; q < per; ++q) {
            const int j = (int)m * per + q;
            if (j >= half) break;
            const int x = 2 * j + p;
            const uint64_t i = site_index(g, x, y, z);
            const uint64_t io = site_index(g, 2 * j + (1 - p), y, z);  // other colour, same column pair
            const int s_old = src[i];
            int n = src[site_index(g, x - 1, y, z)] + src[site_index(g, x + 1, y, z)] +
                    src[site_index(g, x, y - 1, z)] + src[site_index(g, x, y + 1, z)];
            if (g.dims == 3) n += src[site_index(g, x, y, z - 1)] + src[site_index(g, x, y, z + 1)];
            const int k_old = state_of_spin(g.two_S, s_old);
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
            const int s_new = spin_of_state(g.two_S, k_new);
            bool allowed = true;
            if (g.model == LAT_NE) {
                allowed = src[site_index(g, x, y - 1, z)] == 1 && src[site_index(g, x + 1, y, z)] == 1;
            }
            int s_fin = s_old;
            if (allowed) {
                const TabEntry e = stab[(s_new - s_old + g.dsmax) * g.nn + (n + g.nmax)];
                if (e.always || u_acc < e.thr) {
                    s_fin = s_new;
                    if (g.flags != nullptr && s_new != s_old)
                        atomicOr(&g.flags[i >> 5], 1u << (uint32_t)(i & 31));
                }
            }
            dst[i] = (int8_t)s_fin;
            if (colour == 0) dst[io] = src[io];
            if (measure) {
                bond += (long long)s_fin * n;
                const int so = dst[io];
                mag += s_fin + so;
                up += (s_fin > 0) + (so > 0);
                if (g.flags != nullptr) {
                    unfl += ((g.flags[i >> 5] >> (uint32_t)(i & 31)) & 1u) ? 0 : 1;
                    unfl += ((g.flags[io >> 5] >> (uint32_t)(io & 31)) & 1u) ? 0 : 1;
                }
            }
        }
    }
    if (measure) {
        unsigned long long *slot = series_slot(g.ctrl, sweep);
        long long v;
        v = block_sum_ll(bond, red);
        if (threadIdx.x == 0) add_counter(slot + 0, v);
        v = block_sum_ll(mag, red);
        if (threadIdx.x == 0) add_counter(slot + 1, v);
        v = block_sum_ll(up, red);
        if (threadIdx.x == 0) add_counter(slot + 2, v);
        v = block_sum_ll(unfl, red);
        if (threadIdx.x == 0) add_counter(slot + 3, v);
    }
}

// Counters of the current configuration from their definitions (used before
// the first sweep and after set_state).
__global__ void __launch_bounds__(kThreads) k_measure(Geom g, const int8_t *sp, unsigned long long *out)
{
    __shared__ long long red[kThreads / 32];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    long long bond = 0, mag = 0, up = 0, unfl = 0;
    if (i < g.N) {
        const int L = g.L;
        const int x = (int)(i % (uint64_t)L);
        const int y = (int)((i / (uint64_t)L) % (uint64_t)L);
        const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
        const int s = sp[i];
        int nf = sp[site_index(g, x + 1, y, z)] + sp[site_index(g, x, y + 1, z)];
        if (g.dims == 3) nf += sp[site_index(g, x, y, z + 1)];
        bond = (long long)s * nf;
        mag = s;
        up = s > 0;
        if (g.flags != nullptr) unfl = ((g.flags[i >> 5] >> (uint32_t)(i & 31)) & 1u) ? 0 : 1;
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
}

__global__ void k_advance(Ctrl *ctrl, unsigned long long k) { ctrl->sweep += k; }

__global__ void k_set_ctrl(Ctrl *ctrl, unsigned long long sweep, unsigned long long *series,
                           unsigned long long base, unsigned long long cap)
{
    ctrl->sweep = sweep;
    ctrl->series = series;
    ctrl->series_base = base;
    ctrl->series_cap = cap;
}

}  // namespace

cudaError_t launch_init(const Geom &g, int init, double c, cudaStream_t st)
{
    uint32_t thr_c = 0;
    if (init == LAT_INIT_EQUILIBRIUM) {
        // floor(c * 2^32), c in (0, 1): exact in double.
        thr_c = (uint32_t)floor(ldexp(c, 32));
    }
    const uint64_t groups = (g.N + 3) >> 2;
    const unsigned blocks = (unsigned)((groups + kThreads - 1) / kThreads);
    k_init<<<blocks, kThreads, 0, st>>>(g, init, thr_c);
    return cudaGetLastError();
}

cudaError_t launch_half_sweep_generic(const Geom &g, int colour, int off, cudaStream_t st)
{
    const uint64_t total = (uint64_t)g.rows * g.G;
    const unsigned blocks = (unsigned)((total + kThreads - 1) / kThreads);
    const size_t smem = (size_t)g.tab_n * sizeof(TabEntry);
    k_half_sweep<<<blocks, kThreads, smem, st>>>(g, colour, off);
    return cudaGetLastError();
}

cudaError_t launch_measure(const Geom &g, const int8_t *spins, unsigned long long *out4, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((g.N + kThreads - 1) / kThreads);
    k_measure<<<blocks, kThreads, 0, st>>>(g, spins, out4);
    return cudaGetLastError();
}

cudaError_t launch_advance(Ctrl *ctrl, unsigned long long k, cudaStream_t st)
{
    k_advance<<<1, 1, 0, st>>>(ctrl, k);
    return cudaGetLastError();
}

cudaError_t launch_set_ctrl(Ctrl *ctrl, unsigned long long sweep, unsigned long long *series,
                            unsigned long long base, unsigned long long cap, cudaStream_t st)
{
    k_set_ctrl<<<1, 1, 0, st>>>(ctrl, sweep, series, base, cap);
    return cudaGetLastError();
}

}  // namespace lat
