// kernels_rsite.cu -- the paper's own North-East GPU algorithm (§III.B,
// the second algorithm: steps 3-10, Figs. 4-5): random sub-lattices and
// random sites, which keeps the serial relaxation dynamics that the
// checkerboard changes.  2D spin-1/2, either model.
//
// The lattice is cut into Q = (L/b)^2 sub-lattices of P = b*b spins.  One
// sweep is two launches of the sub-lattice kernel plus one measurement
// kernel.  In a launch every sub-lattice is processed once (step 5: each is
// picked by exactly one block, so the block-to-sub-lattice permutation is
// the identity): it is staged in shared memory with its four boundary
// strips and its persistence bytes, makes q rounds of lambda concurrent
// random picks (q * lambda = P/2, steps 6-8) and is written back (step 9).
// The boundary strips keep the values the launch started with.  Launch 0
// reads s[t & 1] and writes the scratch buffer, launch 1 reads the scratch
// buffer and writes s[(t+1) & 1], so no sub-lattice reads a boundary that
// another one is writing.
//
// Thread i of sub-lattice B (row-major) makes one Philox4x32-10 call per
// two rounds: in launch l of sweep t, rounds 2k and 2k+1 share the call with
// counter (B*C + k*lambda + i, t lo, t hi, 4 + l), C = ceil(q/2)*lambda;
// round r takes word 2(r&1) for the site (floor(w * P / 2^32), row-major
// inside the sub-lattice) and word 2(r&1)+1 for the acceptance draw.  Every
// pick of a round is decided from the state at the start of the round; when
// several pick one site the lowest thread index's outcome is kept.  With
// one sub-lattice (b = L) the neighbours wrap inside it, so Q = lambda = 1
// is serial random-site Metropolis.
//
// The balance-preserving variant (after Fig. 5) makes q/2 rounds per
// launch, red (colour 0) and white (colour 1) alternating, each picking
// among the P/2 sites of its colour (m = floor(w * P/2 / 2^32), row m / (b/2),
// column 2 (m mod b/2) + ((row + colour) & 1)), and four launches per sweep
// with tags 4..7; launches 0 and 2 write the scratch buffer, 1 and 3 write
// s[(t+1) & 1].
//
// GPU mapping.  lambda <= 32: a group of lambda lanes owns one sub-lattice,
// a warp holds 32/lambda groups (fewer when shared memory is short) and
// a CTA several independent warps; collisions are resolved in the warp
// with match_any (lowest lane wins).  lambda > 32: one CTA of lambda
// threads per sub-lattice, collisions through an atomicMin owner array.
// The staged sub-lattice is x-fastest with a one-site halo ring, so a
// pick's four neighbours are plain loads at +-1 and +-pitch; rows move
// between it and the planar global layout as 4-byte words interleaved with
// byte permutes.
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kMaxTab = 45;          // 2D spin-1/2 table: (2*2+1) x (2*4+1)
constexpr size_t kWarpBudget = 64 * 1024;   // shared memory per warp group set
constexpr int kMaxWarpsPerCta = 8;

struct RsArgs {
    Geom g;
    int8_t *scratch;    // launch 0 output, launch 1 input
    int b, logb, lambda, loglam, launch, off;
    int balanced, rounds;   // balance-preserving variant; rounds per launch
    int per_warp, warps;    // lambda <= 32: sub-lattices per warp, warps per CTA
    int tile_bytes;         // shared-memory bytes of one staged sub-lattice
};

// One staged sub-lattice, x-fastest with a halo: g[(ly+1)*pitch + 4 + lx]
// for lx, ly in [0, b) (pitch = b + 8, so interior rows start on 4-byte
// boundaries); the north and south halo rows are rows 0 and b+1, the west and
// east halo columns are columns 3 and b+4.  Persistence bytes follow:
// fl[(c*b + ly)*(b/8) + m] for colour c, group m of the row.
struct Tile {
    int8_t *g;
    uint8_t *fl;
    int pitch;
};

LAT_HD size_t grid_bytes_of(int b) { return (((size_t)(b + 2) * (size_t)(b + 8)) + 15) & ~(size_t)15; }
LAT_HD size_t tile_bytes_of(int b) { return grid_bytes_of(b) + (size_t)b * b / 4; }

LAT_D Tile tile_at(unsigned char *base, int b)
{
    Tile t;
    t.g = reinterpret_cast<int8_t *>(base);
    t.fl = base + grid_bytes_of(b);
    t.pitch = b + 8;
    return t;
}

LAT_D uint64_t pidx(const Geom &g, int x, int y)
{
    return (uint64_t)((x + y) & 1) * g.plane + (uint64_t)y * g.half + (uint64_t)(x >> 1);
}

LAT_D int wrapi(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Planar words -> x-fastest words.  A holds 4 colour-0 sites of a row, B the 4
// colour-1 sites of the same 8 columns; on an even row (x0, y0 even) colour
// 0 sits at even x.  lo/hi are the 8 sites in x order.
LAT_D void interleave(uint32_t A, uint32_t B, bool odd_row, uint32_t &lo, uint32_t &hi)
{
    lo = odd_row ? __byte_perm(A, B, 0x1504) : __byte_perm(A, B, 0x5140);
    hi = odd_row ? __byte_perm(A, B, 0x3726) : __byte_perm(A, B, 0x7362);
}

LAT_D void deinterleave(uint32_t lo, uint32_t hi, bool odd_row, uint32_t &A, uint32_t &B)
{
    const uint32_t ev = __byte_perm(lo, hi, 0x6420), od = __byte_perm(lo, hi, 0x7531);
    A = odd_row ? od : ev;
    B = odd_row ? ev : od;
}

// Load planar row y (8-site groups k of the sub-lattice's columns) into the
// tile row `trow` (0 .. b+1).
LAT_D void load_row(const Geom &g, const int8_t *src, const Tile &t, int x0, int y, int trow, int k)
{
    const uint64_t o = (uint64_t)y * g.half + (uint64_t)(x0 >> 1) + 4 * (uint64_t)k;
    const uint32_t A = *reinterpret_cast<const uint32_t *>(src + o);
    const uint32_t B = *reinterpret_cast<const uint32_t *>(src + g.plane + o);
    uint32_t lo, hi;
    interleave(A, B, (y & 1) != 0, lo, hi);
    uint32_t *d = reinterpret_cast<uint32_t *>(t.g + trow * t.pitch + 4 + 8 * k);
    d[0] = lo;
    d[1] = hi;
}

template <bool kNE>
LAT_D void load_tile(const Geom &g, const int8_t *src, const Tile &t, int x0, int y0, int b, bool whole, int tid,
                     int nthr)
{
    const int L = g.L, groups = b >> 3;   // 8-site groups per row
    for (int v = tid; v < b * groups; v += nthr) {
        const int ly = v / groups, k = v - ly * groups;
        load_row(g, src, t, x0, y0 + ly, ly + 1, k);
    }
    if (!whole) {
        const int yn = wrapi(y0 - 1, L), ys = wrapi(y0 + b, L);
        for (int v = tid; v < 2 * groups; v += nthr) {
            const int side = v >= groups, k = v - side * groups;
            load_row(g, src, t, x0, side ? ys : yn, side ? b + 1 : 0, k);
        }
        const int xw = wrapi(x0 - 1, L), xe = wrapi(x0 + b, L);
        for (int v = tid; v < 2 * b; v += nthr) {
            const int side = v >= b, ly = v - side * b;
            t.g[(ly + 1) * t.pitch + (side ? b + 4 : 3)] = src[pidx(g, side ? xe : xw, y0 + ly)];
        }
    }
    if constexpr (kNE) {
        const int fpr = b >> 3;
        for (int v = tid; v < 2 * b * fpr; v += nthr) {
            const int row = v / fpr, m = v - row * fpr, c = row >= b, ly = row - c * b;
            t.fl[v] = g.flags[((uint64_t)c * g.rows + (uint64_t)(y0 + ly)) * g.G + (uint64_t)((x0 >> 3) + m)];
        }
    }
}

// One sub-lattice: the halo ring as the periodic image of the interior
// (called after the interior is loaded and visible to the caller's group).
LAT_D void wrap_halo(const Tile &t, int b, int tid, int nthr)
{
    for (int v = tid; v < 4 * b; v += nthr) {
        const int side = v / b, i = v - side * b;
        if (side == 0) t.g[4 + i] = t.g[b * t.pitch + 4 + i];                           // north <- row b-1
        else if (side == 1) t.g[(b + 1) * t.pitch + 4 + i] = t.g[t.pitch + 4 + i];      // south <- row 0
        else if (side == 2) t.g[(i + 1) * t.pitch + 3] = t.g[(i + 1) * t.pitch + 3 + b]; // west <- col b-1
        else t.g[(i + 1) * t.pitch + 4 + b] = t.g[(i + 1) * t.pitch + 4];                 // east <- col 0
    }
}

template <bool kNE>
LAT_D void store_tile(const Geom &g, int8_t *dst, const Tile &t, int x0, int y0, int b, int tid, int nthr)
{
    const int groups = b >> 3;
    for (int v = tid; v < b * groups; v += nthr) {
        const int ly = v / groups, k = v - ly * groups, y = y0 + ly;
        const uint32_t *s = reinterpret_cast<const uint32_t *>(t.g + (ly + 1) * t.pitch + 4 + 8 * k);
        uint32_t A, B;
        deinterleave(s[0], s[1], (y & 1) != 0, A, B);
        const uint64_t o = (uint64_t)y * g.half + (uint64_t)(x0 >> 1) + 4 * (uint64_t)k;
        *reinterpret_cast<uint32_t *>(dst + o) = A;
        *reinterpret_cast<uint32_t *>(dst + g.plane + o) = B;
    }
    if constexpr (kNE) {
        const int fpr = b >> 3;
        for (int v = tid; v < 2 * b * fpr; v += nthr) {
            const int row = v / fpr, m = v - row * fpr, c = row >= b, ly = row - c * b;
            g.flags[((uint64_t)c * g.rows + (uint64_t)(y0 + ly)) * g.G + (uint64_t)((x0 >> 3) + m)] = t.fl[v];
        }
    }
}

// Decide one pick from the tile as it stands: the site, its new value and
// whether it changes.
// colour < 0: a pick among all P sites; else among the P/2 sites of that
// colour (the balance-preserving variant).
template <bool kNE>
LAT_D void decide(const Geom &g, const Tile &t, const TabEntry *stab, int b, int logb, int colour,
                  uint32_t w_site, uint32_t w_acc, int &site, int8_t &nv, bool &chg)
{
    if (colour < 0) {
        site = (int)(((uint64_t)w_site * (uint64_t)(b * b)) >> 32);
    } else {
        const int m = (int)(((uint64_t)w_site * (uint64_t)(b * b / 2)) >> 32);
        const int row = m >> (logb - 1);
        site = (row << logb) + 2 * (m & ((b >> 1) - 1)) + ((row + colour) & 1);
    }
    const int lx = site & (b - 1), ly = site >> logb;
    const int8_t *c = t.g + (ly + 1) * t.pitch + 4 + lx;
    const int s_old = c[0];
    const int nN = c[-t.pitch], nS = c[t.pitch], nW = c[-1], nE = c[1];
    bool allowed = true;
    if constexpr (kNE) allowed = nN == 1 && nE == 1;   // §III.B: north and east up
    chg = false;
    if (allowed) {
        const TabEntry e = stab[(-2 * s_old + g.dsmax) * g.nn + (nN + nS + nW + nE + g.nmax)];
        chg = e.always || w_acc < e.thr;
    }
    nv = (int8_t)(chg ? -s_old : s_old);
}

// Write a changed site (and, for a whole-lattice tile, its halo images) and
// set its persistence bit.
template <bool kNE>
LAT_D void commit(const Tile &t, int b, int logb, bool whole, int site, int8_t nv)
{
    const int lx = site & (b - 1), ly = site >> logb;
    const int p = t.pitch;
    t.g[(ly + 1) * p + 4 + lx] = nv;
    if (whole) {
        if (ly == 0) t.g[(b + 1) * p + 4 + lx] = nv;
        if (ly == b - 1) t.g[4 + lx] = nv;
        if (lx == 0) t.g[(ly + 1) * p + 4 + b] = nv;
        if (lx == b - 1) t.g[(ly + 1) * p + 3] = nv;
    }
    if constexpr (kNE) {
        const int c = (lx + ly) & 1;   // x0 and y0 are even
        const int byte = (c * b + ly) * (b >> 3) + (lx >> 3);
        uint32_t *w = reinterpret_cast<uint32_t *>(t.fl) + (byte >> 2);
        atomicOr(w, 1u << (8 * (byte & 3) + ((lx >> 1) & 3)));
    }
}

LAT_D void tile_origin(int T, int nt, int logb, int &x0, int &y0)
{
    x0 = (T % nt) << logb;
    y0 = (T / nt) << logb;
}

// lambda <= 32: warps of groups of lambda lanes, one sub-lattice per group.
template <bool kNE>
__global__ void __launch_bounds__(32 * kMaxWarpsPerCta) k_rsite_warp(RsArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ TabEntry stab[kMaxTab];
    const Geom &g = a.g;
    for (int i = threadIdx.x; i < g.tab_n && i < kMaxTab; i += blockDim.x) stab[i] = g.tab[i];
    __syncthreads();

    const int b = a.b, logb = a.logb, P = b * b, L = g.L;
    const int nt = L >> logb, Q = nt * nt;
    const bool whole = nt == 1;
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)a.off;
    // odd launches read the scratch buffer and write s[(t+1) & 1]; even ones
    // write the scratch buffer from s[t & 1] (launch 0) or s[(t+1) & 1]
    const int8_t *src = (a.launch & 1) ? a.scratch : g.s[(sweep + (a.launch ? 1 : 0)) & 1];
    int8_t *dst = (a.launch & 1) ? g.s[(sweep + 1) & 1] : a.scratch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.per_warp;
    const int T0 = (blockIdx.x * a.warps + warp) * S;
    unsigned char *wbase = sm + (size_t)warp * S * a.tile_bytes;

    for (int k = 0; k < S && T0 + k < Q; ++k) {
        int x0, y0;
        tile_origin(T0 + k, nt, logb, x0, y0);
        load_tile<kNE>(g, src, tile_at(wbase + (size_t)k * a.tile_bytes, b), x0, y0, b, whole, lane, 32);
    }
    __syncwarp();
    if (whole) {   // one sub-lattice: its halo is its own periodic image
        wrap_halo(tile_at(wbase, b), b, lane, 32);
        __syncwarp();
    }

    const int grp = lane >> a.loglam, me = lane & (a.lambda - 1);
    const bool act = grp < S && T0 + grp < Q;
    const int T = T0 + grp;
    const Tile t = tile_at(wbase + (size_t)(act ? grp : 0) * a.tile_bytes, b);
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const int q = a.rounds;
    const uint32_t calls = (uint32_t)((q + 1) >> 1) << a.loglam;   // Philox calls per sub-lattice
    const uint32_t base = (uint32_t)T * calls + (uint32_t)me;
    const uint32_t tag = 4u + (uint32_t)a.launch;
    auto round = [&](uint32_t w_site, uint32_t w_acc, int colour) {
        int key = -1 - lane;   // distinct for idle lanes
        int site = 0;
        int8_t nv = 0;
        bool chg = false;
        if (act) {
            decide<kNE>(g, t, stab, b, logb, colour, w_site, w_acc, site, nv, chg);
            key = grp * P + site;
        }
        __syncwarp();                        // every read of the round is done
        const unsigned m = __match_any_sync(0xffffffffu, key);
        if (act && chg && (__ffs(m) - 1) == lane) commit<kNE>(t, b, logb, whole, site, nv);
        __syncwarp();
    };
    for (int r = 0; r < q; r += 2) {
        U4 w = U4{0u, 0u, 0u, 0u};
        if (act) w = philox_item(pp, base + ((uint32_t)(r >> 1) << a.loglam), tag);
        round(w.x, w.y, a.balanced ? 0 : -1);
        if (r + 1 < q) round(w.z, w.w, a.balanced ? 1 : -1);
    }

    for (int k = 0; k < S && T0 + k < Q; ++k) {
        int xk, yk;
        tile_origin(T0 + k, nt, logb, xk, yk);
        store_tile<kNE>(g, dst, tile_at(wbase + (size_t)k * a.tile_bytes, b), xk, yk, b, lane, 32);
    }
}

// lambda > 32: one CTA of lambda threads per sub-lattice.
template <bool kNE>
__global__ void __launch_bounds__(1024) k_rsite_block(RsArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ TabEntry stab[kMaxTab];
    const Geom &g = a.g;
    const int b = a.b, logb = a.logb, P = b * b, L = g.L;
    const int nt = L >> logb;
    const bool whole = nt == 1;
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)a.off;
    // odd launches read the scratch buffer and write s[(t+1) & 1]; even ones
    // write the scratch buffer from s[t & 1] (launch 0) or s[(t+1) & 1]
    const int8_t *src = (a.launch & 1) ? a.scratch : g.s[(sweep + (a.launch ? 1 : 0)) & 1];
    int8_t *dst = (a.launch & 1) ? g.s[(sweep + 1) & 1] : a.scratch;
    const int T = blockIdx.x;
    int x0, y0;
    tile_origin(T, nt, logb, x0, y0);
    const Tile t = tile_at(sm, b);
    uint32_t *own = reinterpret_cast<uint32_t *>(sm + a.tile_bytes);   // P entries

    for (int i = threadIdx.x; i < g.tab_n && i < kMaxTab; i += blockDim.x) stab[i] = g.tab[i];
    load_tile<kNE>(g, src, t, x0, y0, b, whole, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < P; i += blockDim.x) own[i] = 0xFFFFFFFFu;
    __syncthreads();
    if (whole) {
        wrap_halo(t, b, threadIdx.x, blockDim.x);
        __syncthreads();
    }

    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const int me = threadIdx.x;
    const int q = a.rounds;
    const uint32_t calls = (uint32_t)((q + 1) >> 1) << a.loglam;
    const uint32_t base = (uint32_t)T * calls + (uint32_t)me;
    const uint32_t tag = 4u + (uint32_t)a.launch;
    auto round = [&](uint32_t w_site, uint32_t w_acc, int colour) {
        int site;
        int8_t nv;
        bool chg;
        decide<kNE>(g, t, stab, b, logb, colour, w_site, w_acc, site, nv, chg);
        __syncthreads();                     // every read of the round is done
        atomicMin(&own[site], (uint32_t)me);
        __syncthreads();
        if (chg && own[site] == (uint32_t)me) commit<kNE>(t, b, logb, whole, site, nv);
        __syncthreads();                     // writes done before the reset and the next reads
        own[site] = 0xFFFFFFFFu;
    };
    for (int r = 0; r < q; r += 2) {
        const U4 w = philox_item(pp, base + ((uint32_t)(r >> 1) << a.loglam), tag);
        round(w.x, w.y, a.balanced ? 0 : -1);
        if (r + 1 < q) round(w.z, w.w, a.balanced ? 1 : -1);
    }
    __syncthreads();
    store_tile<kNE>(g, dst, t, x0, y0, b, threadIdx.x, blockDim.x);
}

// Counters of the state after the sweep (the sub-lattices of launch 1 cannot
// see their neighbours' final values), word-wise on the +-1 bytes of the
// planar layout: a thread takes W 4-byte words of colour 1 in row y (4W
// sites) and the colour-0 words at the same indexes.  Byte bit 1 marks a
// down spin (0x01 up, 0xFF down): the bond of a colour-1 site is 4 - 2 *
// (# unlike neighbours), and every bond has exactly one colour-1 end.
constexpr int kMeasThreads = 256;

LAT_D int byte_sum(uint32_t x)
{
    const uint32_t s = (x & 0x00FF00FFu) + ((x >> 8) & 0x00FF00FFu);
    return (int)((s & 0xFFFFu) + (s >> 16));
}

template <int W>
__global__ void __launch_bounds__(kMeasThreads) k_rsite_measure(Geom g, int off)
{
    __shared__ long long red[kMeasThreads / 32];
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const int8_t *sp = g.s[(sweep + 1) & 1];
    const uint32_t nwr = g.half >> 2;              // words per plane row
    const uint32_t cpr = nwr / W;                  // chunks per plane row
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    long long bond = 0, mag = 0, up = 0, unfl = 0, acf = 0;
    if (t < (uint64_t)g.L * cpr) {
        const int L = g.L;
        const int y = (int)(t / cpr), k = (int)(t % cpr);
        const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
        const uint32_t *p0 = reinterpret_cast<const uint32_t *>(sp);
        const uint32_t *p1 = reinterpret_cast<const uint32_t *>(sp + g.plane);
        const uint64_t r0 = (uint64_t)y * nwr, rm = (uint64_t)ym * nwr, rp = (uint64_t)yp * nwr;
        uint32_t S[W], O[W], U[W], D[W], Lf[W], R[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            S[w] = p1[r0 + W * k + w];
            O[w] = p0[r0 + W * k + w];
            U[w] = p0[rm + W * k + w];
            D[w] = p0[rp + W * k + w];
        }
        // colour-1 site j sits at x = 2j + ((1 + y) & 1): its row neighbours
        // are colour-0 sites j-1, j (odd x... even x) or j, j+1
        const bool right = ((1 + y) & 1) != 0;
        const uint32_t adj = p0[r0 + wrap_once(right ? W * k + W : W * k + nwr - 1, nwr)];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (!right) {   // west is j-1, east is j
                Lf[w] = __funnelshift_l(w == 0 ? adj : O[w - 1], O[w], 8);
                R[w] = O[w];
            } else {        // west is j, east is j+1
                Lf[w] = O[w];
                R[w] = __funnelshift_r(O[w], w == W - 1 ? adj : O[w + 1], 8);
            }
        }
        const uint32_t M1 = 0x02020202u;
        uint32_t ue = 0, dn = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ue += ((U[w] ^ S[w]) & M1) + ((D[w] ^ S[w]) & M1) + ((Lf[w] ^ S[w]) & M1) + ((R[w] ^ S[w]) & M1);
            dn += (S[w] & M1) + (O[w] & M1);
        }
        const int d2 = byte_sum(dn);
        bond = 16 * W - byte_sum(ue);
        mag = 8 * W - d2;
        up = 8 * W - (d2 >> 1);
        if (g.flags != nullptr) {   // one byte per 4-site group, bit q = site 4m+q ever changed
            const uint8_t *f1 = g.flags + ((uint64_t)g.rows + (uint64_t)y) * g.G + (uint64_t)(W * k);
            const uint8_t *f0 = g.flags + (uint64_t)y * g.G + (uint64_t)(W * k);
            int ch = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) ch += __popc((uint32_t)f1[w] & 0xFu) + __popc((uint32_t)f0[w] & 0xFu);
            unfl = 8 * W - ch;
        }
        if (g.ref != nullptr) {
            const uint32_t *q0 = reinterpret_cast<const uint32_t *>(g.ref);
            const uint32_t *q1 = reinterpret_cast<const uint32_t *>(g.ref + g.plane);
            uint32_t dr = 0;
#pragma unroll
            for (int w = 0; w < W; ++w)
                dr += ((S[w] ^ q1[r0 + W * k + w]) & M1) + ((O[w] ^ q0[r0 + W * k + w]) & M1);
            acf = 8 * W - byte_sum(dr);
        }
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

int log2i(int v) { return 31 - __builtin_clz((unsigned)v); }

// Launch geometry: shared memory per CTA and the grid.
struct RsPlan {
    int per_warp, warps, threads, blocks;
    size_t smem;
};

RsPlan plan(int L, int b, int lambda)
{
    RsPlan p;
    const size_t tb = tile_bytes_of(b);
    const int Q = (L / b) * (L / b);
    if (lambda <= 32) {
        int S = 32 / lambda;
        const int fit = (int)(kWarpBudget / tb);
        if (S > fit) S = fit > 0 ? fit : 1;
        int W = (int)(kWarpBudget / (tb * (size_t)S));
        W = W < 1 ? 1 : (W > kMaxWarpsPerCta ? kMaxWarpsPerCta : W);
        const int per_cta = S * W;
        if (per_cta > Q) W = (Q + S - 1) / S;   // small lattices: no idle warps
        p.per_warp = S;
        p.warps = W;
        p.threads = 32 * W;
        p.blocks = (Q + S * W - 1) / (S * W);
        p.smem = tb * (size_t)S * (size_t)W;
    } else {
        p.per_warp = 1;
        p.warps = lambda / 32;
        p.threads = lambda;
        p.blocks = Q;
        p.smem = tb + 4 * (size_t)b * b;   // tile + owner array
    }
    return p;
}

}  // namespace

bool rsite_params_ok(const Geom &g, int b, int lambda, bool balanced)
{
    if (g.dims != 2 || g.two_S != 1 || g.bits[0] != nullptr || g.cpl != nullptr || g.tab_n > kMaxTab ||
        g.model == LAT_POTTS)
        return false;
    if (b < 8 || b > 256 || (b & (b - 1)) != 0 || (g.L % b) != 0) return false;
    const int half_p = b * b / 2;
    if (lambda < 1 || lambda > 1024 || (lambda & (lambda - 1)) != 0 || lambda > half_p) return false;
    if (balanced && ((half_p / lambda) % 4) != 0) return false;   // q/2 rounds per launch, q/2 even
    return plan(g.L, b, lambda).smem <= 200 * 1024;
}

cudaError_t launch_sweep_rsite(const Geom &g, int8_t *scratch, int b, int lambda, bool balanced, int off,
                               cudaStream_t st)
{
    const RsPlan p = plan(g.L, b, lambda);
    RsArgs a;
    a.g = g;
    a.scratch = scratch;
    a.b = b;
    a.logb = log2i(b);
    a.lambda = lambda;
    a.loglam = log2i(lambda);
    a.off = off;
    a.per_warp = p.per_warp;
    a.warps = p.warps;
    a.tile_bytes = (int)tile_bytes_of(b);
    a.balanced = balanced ? 1 : 0;
    const int q = (b * b / 2) / lambda;
    a.rounds = balanced ? q / 2 : q;
    static bool attr = false;
    if (!attr) {
        const int lim = 200 * 1024;
        cudaError_t e = cudaFuncSetAttribute(k_rsite_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_rsite_warp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_rsite_block<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_rsite_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const bool ne = g.model == LAT_NE;
    for (int launch = 0; launch < (balanced ? 4 : 2); ++launch) {
        a.launch = launch;
        if (lambda <= 32) {
            if (ne) k_rsite_warp<true><<<p.blocks, p.threads, p.smem, st>>>(a);
            else k_rsite_warp<false><<<p.blocks, p.threads, p.smem, st>>>(a);
        } else {
            if (ne) k_rsite_block<true><<<p.blocks, p.threads, p.smem, st>>>(a);
            else k_rsite_block<false><<<p.blocks, p.threads, p.smem, st>>>(a);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // 16 sites per measuring thread when rows hold whole 4-word chunks (L % 32 == 0), else 4
    const uint64_t words = (uint64_t)g.L * (g.half >> 2);
    if ((g.half >> 2) % 4 == 0) {
        const uint64_t n = words / 4;
        k_rsite_measure<4><<<(unsigned)((n + kMeasThreads - 1) / kMeasThreads), kMeasThreads, 0, st>>>(g, off);
    } else {
        k_rsite_measure<1><<<(unsigned)((words + kMeasThreads - 1) / kMeasThreads), kMeasThreads, 0, st>>>(g, off);
    }
    return cudaGetLastError();
}

}  // namespace lat
