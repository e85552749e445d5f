// kernels_rsite.cu -- the paper's own North-East GPU algorithm (§III.B,
// the second algorithm: steps 3-10, Figs. 4-5): random sub-lattices and
// random sites, which keeps the serial relaxation dynamics that the
// checkerboard changes.  2D spin-1/2, either model.
//
// The lattice is cut into Q = (L/b)^2 sub-lattices of P = b*b spins.  One
// sweep is two launches of k_rsite plus one measurement kernel.  In a launch
// one CTA owns one sub-lattice (step 5: every sub-lattice is picked by
// exactly one block, so the block-to-sub-lattice permutation is the
// identity): it stages the sub-lattice, its four boundary strips and its
// persistence bytes in shared memory, runs q rounds of lambda concurrent
// random picks (q * lambda = P/2, steps 6-8) and writes the sub-lattice
// back (step 9).  The boundary strips keep the values the launch started
// with.  Launch 0 reads s[t & 1] and writes the scratch buffer, launch 1
// reads the scratch buffer and writes s[(t+1) & 1], so no CTA reads a
// boundary another CTA is writing.
//
// Pick p = r*lambda + i of launch l in sweep t of sub-lattice B draws
// Philox4x32-10 with counter (B*P/2 + p, t lo, t hi, 4 + l): word 0 picks
// the site (floor(w0 * P / 2^32), row-major in the sub-lattice), word 1 is
// the acceptance draw.  Every pick of a round is decided from the state at
// the start of the round; when several pick one site the lowest thread
// index's outcome is kept.  With one sub-lattice (b = L) the neighbours
// wrap inside it, so Q = lambda = 1 is serial random-site Metropolis.
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kMaxTab = 45;    // 2D spin-1/2 table: (2*2+1) x (2*4+1)

struct RsArgs {
    Geom g;
    int8_t *scratch;   // launch 0 output, launch 1 input
    int b, logb, lambda, launch, off;
};

LAT_D uint64_t pidx(const Geom &g, int x, int y)
{
    return (uint64_t)((x + y) & 1) * g.plane + (uint64_t)y * g.half + (uint64_t)(x >> 1);
}

LAT_D int wrapi(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Shared memory: [owner: P x u32 when lambda > 32][tile: P][N, S, W, E
// strips: 4b][persistence bytes: b*b/4].
size_t rsite_smem(int b, int lambda)
{
    const size_t P = (size_t)b * b;
    return (lambda > 32 ? 4 * P : 0) + P + 4 * (size_t)b + P / 4;
}

template <bool kNE>
__global__ void __launch_bounds__(1024) k_rsite(RsArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ TabEntry stab[kMaxTab];
    const Geom &g = a.g;
    const int b = a.b, logb = a.logb, P = b * b, L = g.L;
    const bool multi = a.lambda > 32;
    uint32_t *own = reinterpret_cast<uint32_t *>(sm);
    int8_t *tile = reinterpret_cast<int8_t *>(sm + (multi ? 4 * (size_t)P : 0));
    int8_t *bn = tile + P, *bs = bn + b, *bw = bs + b, *be = bw + b;
    uint32_t *fl = reinterpret_cast<uint32_t *>(be + b);   // b*b/4 bytes, 4-byte aligned
    uint8_t *fl8 = reinterpret_cast<uint8_t *>(fl);
    const int fpr = b >> 3;                               // persistence bytes per (colour, row)

    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)a.off;
    const int nt = L >> logb;
    const int B = blockIdx.x;
    const int x0 = (B % nt) << logb, y0 = (B / nt) << logb;
    const int8_t *src = a.launch == 0 ? g.s[sweep & 1] : a.scratch;
    int8_t *dst = a.launch == 0 ? a.scratch : g.s[(sweep + 1) & 1];
    const bool whole = nt == 1;

    for (int i = threadIdx.x; i < g.tab_n && i < kMaxTab; i += blockDim.x) stab[i] = g.tab[i];
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        tile[i] = src[pidx(g, x0 + (i & (b - 1)), y0 + (i >> logb))];
    if (!whole) {
        for (int i = threadIdx.x; i < b; i += blockDim.x) {
            bn[i] = src[pidx(g, x0 + i, wrapi(y0 - 1, L))];
            bs[i] = src[pidx(g, x0 + i, wrapi(y0 + b, L))];
            bw[i] = src[pidx(g, wrapi(x0 - 1, L), y0 + i)];
            be[i] = src[pidx(g, wrapi(x0 + b, L), y0 + i)];
        }
    }
    if constexpr (kNE) {
        for (int i = threadIdx.x; i < 2 * b * fpr; i += blockDim.x) {
            const int c = i / (b * fpr), rem = i - c * b * fpr, ly = rem / fpr, m = rem - ly * fpr;
            fl8[i] = g.flags[((uint64_t)c * g.rows + (uint64_t)(y0 + ly)) * g.G + (uint64_t)((x0 >> 3) + m)];
        }
    }
    if (multi)
        for (int i = threadIdx.x; i < P; i += blockDim.x) own[i] = 0xFFFFFFFFu;
    __syncthreads();

    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const int lane = threadIdx.x & 31;
    const int me = threadIdx.x;
    const bool act = me < a.lambda;
    const int q = (P >> 1) / a.lambda;
    const uint32_t base = (uint32_t)B * (uint32_t)(P >> 1);
    const uint32_t tag = 4u + (uint32_t)a.launch;
    for (int r = 0; r < q; ++r) {
        int site = P + lane;   // out of range: never matches a real pick
        int8_t nv = 0;
        bool chg = false;
        if (act) {
            const U4 w = philox_item(pp, base + (uint32_t)(r * a.lambda + me), tag);
            site = (int)(((uint64_t)w.x * (uint64_t)P) >> 32);
            const int lx = site & (b - 1), ly = site >> logb;
            const int s_old = tile[site];
            const int nN = ly > 0 ? tile[site - b] : (whole ? tile[site + P - b] : bn[lx]);
            const int nS = ly < b - 1 ? tile[site + b] : (whole ? tile[site - P + b] : bs[lx]);
            const int nW = lx > 0 ? tile[site - 1] : (whole ? tile[site + b - 1] : bw[ly]);
            const int nE = lx < b - 1 ? tile[site + 1] : (whole ? tile[site - b + 1] : be[ly]);
            bool allowed = true;
            if constexpr (kNE) allowed = nN == 1 && nE == 1;   // §III.B: north and east up
            if (allowed) {
                const int n = nN + nS + nW + nE;
                const TabEntry e = stab[(-2 * s_old + g.dsmax) * g.nn + (n + g.nmax)];
                chg = e.always || w.y < e.thr;
            }
            nv = (int8_t)(chg ? -s_old : s_old);
        }
        bool win;
        if (!multi) {
            // one warp: the lowest lane among those that picked the site wins
            __syncwarp();
            const unsigned m = __match_any_sync(0xffffffffu, site);
            win = act && (__ffs(m) - 1) == lane;
        } else {
            __syncthreads();                   // every read of the round is done
            if (act) atomicMin(&own[site], (uint32_t)me);
            __syncthreads();
            win = act && own[site] == (uint32_t)me;
        }
        if (win && chg) {
            tile[site] = nv;
            if constexpr (kNE) {
                const int lx = site & (b - 1), ly = site >> logb;
                const int c = (x0 + lx + y0 + ly) & 1;
                const int byte = (c * b + ly) * fpr + (lx >> 3);
                atomicOr(&fl[byte >> 2], 1u << (8 * (byte & 3) + ((lx >> 1) & 3)));
            }
        }
        if (!multi) {
            __syncwarp();
        } else {
            __syncthreads();                   // writes done before the reset and the next reads
            if (act) own[site] = 0xFFFFFFFFu;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        dst[pidx(g, x0 + (i & (b - 1)), y0 + (i >> logb))] = tile[i];
    if constexpr (kNE) {
        for (int i = threadIdx.x; i < 2 * b * fpr; i += blockDim.x) {
            const int c = i / (b * fpr), rem = i - c * b * fpr, ly = rem / fpr, m = rem - ly * fpr;
            g.flags[((uint64_t)c * g.rows + (uint64_t)(y0 + ly)) * g.G + (uint64_t)((x0 >> 3) + m)] = fl8[i];
        }
    }
}

// Counters of the state after the sweep (the tiles of launch 1 cannot see
// their neighbours' final values): thread = one planar index j of row y,
// i.e. one colour-1 site and the colour-0 site beside it.
constexpr int kMeasThreads = 256;

__global__ void __launch_bounds__(kMeasThreads) k_rsite_measure(Geom g, int off)
{
    __shared__ long long red[kMeasThreads / 32];
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const int8_t *sp = g.s[(sweep + 1) & 1];
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    long long bond = 0, mag = 0, up = 0, unfl = 0, acf = 0;
    if (t < (uint64_t)g.L * g.half) {
        const int L = g.L;
        const int y = (int)(t / g.half), j = (int)(t % g.half);
        const int x1 = 2 * j + ((1 + y) & 1);                 // the colour-1 site
        const int s1 = sp[g.plane + (uint64_t)y * g.half + j];
        const int s0 = sp[(uint64_t)y * g.half + j];
        const int n = sp[pidx(g, wrapi(x1 - 1, L), y)] + sp[pidx(g, wrapi(x1 + 1, L), y)] +
                      sp[pidx(g, x1, wrapi(y - 1, L))] + sp[pidx(g, x1, wrapi(y + 1, L))];
        bond = (long long)s1 * n;
        mag = s1 + s0;
        up = (s1 > 0) + (s0 > 0);
        if (g.flags != nullptr) {
            const uint64_t gb = (uint64_t)y * g.G + (uint64_t)(j >> 2);
            const int q = j & 3;
            unfl = (((g.flags[(uint64_t)g.rows * g.G + gb] >> q) & 1) == 0) + (((g.flags[gb] >> q) & 1) == 0);
        }
        if (g.ref != nullptr)
            acf = s1 * g.ref[g.plane + (uint64_t)y * g.half + j] + s0 * g.ref[(uint64_t)y * g.half + j];
    }
    unsigned long long *slot = series_slot(g.ctrl, sweep);
    long long v = block_sum_ll(bond, red);
    if (threadIdx.x == 0) add_counter(slot + 0, v);
    v = block_sum_ll(mag, red);
    if (threadIdx.x == 0) add_counter(slot + 1, v);
    v = block_sum_ll(up, red);
    if (threadIdx.x == 0) add_counter(slot + 2, v);
    if (g.flags != nullptr) {
        v = block_sum_ll(unfl, red);
        if (threadIdx.x == 0) add_counter(slot + 3, v);
    }
    if (g.ref != nullptr) {
        v = block_sum_ll(acf, red);
        if (threadIdx.x == 0) add_counter(acf_slot(g.ctrl, sweep), v);
    }
}

}  // namespace

bool rsite_params_ok(const Geom &g, int b, int lambda)
{
    if (g.dims != 2 || g.two_S != 1 || g.bits[0] != nullptr || g.tab_n > kMaxTab) return false;
    if (b < 8 || b > 256 || (b & (b - 1)) != 0 || (g.L % b) != 0) return false;
    const int half_p = b * b / 2;
    if (lambda < 1 || lambda > 1024 || (lambda & (lambda - 1)) != 0 || lambda > half_p) return false;
    return rsite_smem(b, lambda) <= 200 * 1024;
}

cudaError_t launch_sweep_rsite(const Geom &g, int8_t *scratch, int b, int lambda, int off, cudaStream_t st)
{
    RsArgs a;
    a.g = g;
    a.scratch = scratch;
    a.b = b;
    a.logb = 31 - __builtin_clz((unsigned)b);
    a.lambda = lambda;
    a.off = off;
    const size_t smem = rsite_smem(b, lambda);
    static bool attr[2] = {false, false};
    const int m = g.model == LAT_NE ? 1 : 0;
    if (!attr[m]) {
        cudaError_t e = m ? cudaFuncSetAttribute(k_rsite<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
                          : cudaFuncSetAttribute(k_rsite<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr[m] = true;
    }
    const int tiles = (g.L / b) * (g.L / b);
    const int threads = lambda > 32 ? lambda : 32;
    for (int launch = 0; launch < 2; ++launch) {
        a.launch = launch;
        if (m) k_rsite<true><<<tiles, threads, smem, st>>>(a);
        else k_rsite<false><<<tiles, threads, smem, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const uint64_t n = (uint64_t)g.L * g.half;
    k_rsite_measure<<<(unsigned)((n + kMeasThreads - 1) / kMeasThreads), kMeasThreads, 0, st>>>(g, off);
    return cudaGetLastError();
}

}  // namespace lat
