// kernels_tiled.cu -- one launch per sweep for 2D spin-1/2 lattices (Ising
// and North-East), int8 spins of +-1, L a multiple of 16.
//
// The paper's GPU sweep (§III.A steps 5-8, Fig. 2) copies each sub-lattice
// with its boundary into shared memory, updates the red+blue sites, ends the
// kernel as a device-wide barrier, and relaunches for green+white: two
// launches and two passes over memory per sweep.  Here one launch does the
// whole sweep: each CTA stages a tile of 256 columns x tile_h rows plus a
// two-row / one-word halo in shared memory, updates colour 0 on the tile
// AND on the one-site ring around it (recomputing the ring is legal because
// every draw is keyed by site group and sweep, so the ring holds bit for
// bit what the neighbouring tile computes), then updates colour 1 on the
// tile and writes it to the other spin buffer.  Memory traffic is one read
// and one write per site per sweep (plus the halo).
//
// Work item = one 8-byte word of a row: the four sites of the active colour
// (bytes p, p+2, p+4, p+6, p = (colour + y) & 1) = one Philox call.  A warp
// owns one tile row (32 words), so p is warp-uniform and the neighbour bytes
// are gathered with byte permutes.  Bytes are 0x01 (+1) or 0xFF (-1), so
// bits 1..7 of a byte all equal "spin down"; the number of down neighbours
// is formed for four sites at once with a bit-sliced adder, and a scaled
// table index is assembled with masks only.  The acceptance table is held
// as t' = thr - 1 (all ones = accept without a draw), so a move is accepted
// iff u <= t'; lattices whose table has a never-accept entry (thr = 0,
// possible only for dE/T > 22) use the generic kernel instead.  The Philox
// call is skipped when none of the four sites needs a draw.
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kTileW = 256;         // columns (bytes) per tile = 32 words
constexpr int kWords = kTileW / 8;  // words per tile row (one per lane)
constexpr int kPitch = kWords + 4;  // smem words per row: pad, halo, 32 words, halo, pad
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxTileH = 64;
constexpr int kDefTileH = 64;

struct TiledArgs {
    Geom g;
    int tile_h;
    int off;  // sweep offset relative to ctrl->sweep
};

LAT_D uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) { return __byte_perm(a, b, sel); }

// Byte permute in PTX's generic mode, where bit 3 of a selector nibble
// replicates the sign bit of the selected byte over the output byte
// (__byte_perm uses only the low three bits of each nibble).
LAT_D uint32_t prmt_sign(uint32_t a, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(a), "r"(sel));
    return r;
}

struct Tile {
    uint2 *w;  // [(tile_h + 4) * kPitch]; word (ry, wx) at (ry+2)*kPitch + wx + 2
    LAT_D uint2 &at(int ry, int wx) const { return w[(ry + 2) * kPitch + wx + 2]; }
};

struct Counters {
    int bond = 0, mag = 0, up = 0, unfl = 0;
};

// Gather the four sites of parity P of word (ry, wx) and their four
// neighbours into 4-byte words (byte q <-> site q at byte P + 2q).
template <int P>
LAT_D void gather(const Tile &t, int ry, int wx, uint2 &W, uint32_t &S, uint32_t &U, uint32_t &D,
                  uint32_t &Lf, uint32_t &R)
{
    W = t.at(ry, wx);
    const uint2 Wu = t.at(ry - 1, wx);
    const uint2 Wd = t.at(ry + 1, wx);
    if (P == 0) {
        // sites at bytes 0,2,4,6; left = byte 7 of the previous word, 1, 3, 5; right = 1,3,5,7
        const uint32_t wl = t.at(ry, wx - 1).y;
        S = prmt(W.x, W.y, 0x6420u);
        U = prmt(Wu.x, Wu.y, 0x6420u);
        D = prmt(Wd.x, Wd.y, 0x6420u);
        R = prmt(W.x, W.y, 0x7531u);
        Lf = prmt(wl, prmt(W.x, W.y, 0x0531u), 0x6543u);
    } else {
        // sites at bytes 1,3,5,7; left = 0,2,4,6; right = 2,4,6, byte 0 of the next word
        const uint32_t wr = t.at(ry, wx + 1).x;
        S = prmt(W.x, W.y, 0x7531u);
        U = prmt(Wu.x, Wu.y, 0x7531u);
        D = prmt(Wd.x, Wd.y, 0x7531u);
        Lf = prmt(W.x, W.y, 0x6420u);
        R = prmt(Lf, wr, 0x4321u);
    }
}

// Spread a 4-bit per-site mask to the 8 flag bits of a word (site q of
// parity P sits at byte P + 2q).
template <int P>
LAT_D uint32_t spread_flags(uint32_t a4)
{
    const uint32_t s = (a4 & 1u) | ((a4 & 2u) << 1) | ((a4 & 4u) << 2) | ((a4 & 8u) << 3);
    return s << P;
}

// Update one work item and return the new word.  flags: in, the word's
// persistence byte; out, with this pass's flips added (North-East).
// kMeasure (colour-1 pass): accumulate the counters of the final word.
template <bool kNE, int P, bool kMeasure>
LAT_D uint2 update(const Tile &t, const uint32_t *sthr, const Geom &g, int ry, int wx, uint32_t grp,
                   uint32_t ctr1, uint32_t ctr2, uint32_t colour, uint32_t &flags, Counters &cnt)
{
    uint2 W;
    uint32_t S, U, D, Lf, R;
    gather<P>(t, ry, wx, W, S, U, D, Lf, R);
    // Bit-sliced count (b2 b1 b0) of down neighbours, valid in bits 1..7 of each byte.
    const uint32_t s1 = U ^ D ^ Lf;
    const uint32_t c1 = (U & D) | (U & Lf) | (D & Lf);
    const uint32_t b0 = s1 ^ R;
    const uint32_t b1 = c1 ^ (s1 & R);
    const uint32_t b2 = c1 & s1 & R;
    // Byte offset into the 16-entry table (index sd<<3 | nd, 4 bytes each):
    // bit 2 = b0, bit 3 = b1, bit 4 = b2, bit 5 = sd.  Every bit 1..7 of a
    // byte carries the same flag, so masks alone place them.
    const uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) |
                         (S & 0x20202020u);
    const char *tb = reinterpret_cast<const char *>(sthr);
    uint32_t t0 = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
    uint32_t t1 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
    uint32_t t2 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
    uint32_t t3 = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
    uint32_t locked = 0;
    if (kNE) {
        // §III.B: a site may change only if north (U) and east (R) are up.
        // Sign-replicating each byte of (U | R) gives an all-ones mask for a
        // locked site: it then needs no draw, and its flip is masked off.
        locked = U | R;
        t0 |= prmt_sign(locked, 0x8888u);
        t1 |= prmt_sign(locked, 0x9999u);
        t2 |= prmt_sign(locked, 0xAAAAu);
        t3 |= prmt_sign(locked, 0xBBBBu);
    }
    uint32_t acc = 0xFu;
    if (min(min(t0, t1), min(t2, t3)) != 0xFFFFFFFFu) {
        const U4 u = philox(U4{grp, ctr1, ctr2, colour}, g.key0, g.key1);
        acc = (u.x <= t0 ? 1u : 0u) | (u.y <= t1 ? 2u : 0u) | (u.z <= t2 ? 4u : 0u) |
              (u.w <= t3 ? 8u : 0u);
    }
    // Byte mask 0xFE at each flipped site: +1 (0x01) <-> -1 (0xFF).
    uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu;
    if (kNE) {
        F &= ~locked;
        const uint32_t a4 = ((((F >> 1) & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
        flags |= spread_flags<P>(a4);
    }
    uint2 Wn;
    if (P == 0) {
        Wn.x = W.x ^ prmt(F, 0u, 0x4140u);
        Wn.y = W.y ^ prmt(F, 0u, 0x4342u);
    } else {
        Wn.x = W.x ^ prmt(F, 0u, 0x1404u);
        Wn.y = W.y ^ prmt(F, 0u, 0x3424u);
    }
    if (kMeasure) {
        // Bond sum over this word's colour-1 sites: s' * (sum of its four
        // colour-0 neighbours) = 2 * (# equal neighbours) - 4 per site.
        const uint32_t Sn = S ^ F;
        const uint32_t M1 = 0x02020202u;
        const int eq = __popc(~(Sn ^ U) & M1) + __popc(~(Sn ^ D) & M1) +
                       __popc(~(Sn ^ Lf) & M1) + __popc(~(Sn ^ R) & M1);
        cnt.bond += 2 * eq - 16;
        const int downs = __popc(Wn.x & M1) + __popc(Wn.y & M1);
        cnt.mag += 8 - 2 * downs;
        cnt.up += 8 - downs;
        if (kNE) cnt.unfl += 8 - __popc(flags);
    }
    return Wn;
}

LAT_D int wrap(int v, int n)
{
    v += (v < 0) ? n : 0;
    v -= (v >= n) ? n : 0;
    return v;
}

template <bool kNE>
__global__ void __launch_bounds__(kThreads) k_sweep_tiled(TiledArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t sthr[16];
    __shared__ int red[kWarps][4];

    const Geom &g = a.g;
    const int L = g.L;
    const int wpr = L >> 3;  // words per lattice row (= Philox groups per row)
    const int x0 = blockIdx.x * kTileW;
    const int y0 = blockIdx.y * a.tile_h;
    const int nw = min(kWords, (L - x0) >> 3);
    const int th = min(a.tile_h, L - y0);
    const int w0 = x0 >> 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    Tile t;
    t.w = reinterpret_cast<uint2 *>(smem_raw);
    uint8_t *sflag = smem_raw + (size_t)(a.tile_h + 4) * kPitch * sizeof(uint2);  // [tile_h][32]

    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)a.off;
    const int8_t *src = g.s[sweep & 1];
    int8_t *dst = g.s[(sweep + 1) & 1];
    const uint32_t ctr1 = (uint32_t)sweep, ctr2 = (uint32_t)(sweep >> 32);

    // ---- stage rows y0-2 .. y0+th+1: 16-byte interior loads, 8-byte halo words
    const int rows = th + 4;
    const int n16 = nw >> 1;  // 16-byte chunks per row
    for (int i = threadIdx.x; i < rows * 16; i += kThreads) {
        const int r = i >> 4, c = i & 15;
        if (c >= n16) continue;
        const int gy = wrap(y0 + r - 2, L);
        const uint4 v = *reinterpret_cast<const uint4 *>(src + (size_t)gy * L + x0 + 16 * c);
        *reinterpret_cast<uint4 *>(&t.at(r - 2, 2 * c)) = v;
    }
    for (int i = threadIdx.x; i < rows * 2; i += kThreads) {
        const int r = i >> 1, side = i & 1;
        const int gy = wrap(y0 + r - 2, L);
        const int gw = wrap(side ? w0 + nw : w0 - 1, wpr);
        t.at(r - 2, side ? nw : -1) =
            *reinterpret_cast<const uint2 *>(src + (size_t)gy * L + 8 * (size_t)gw);
    }
    if (kNE) {
        const uint8_t *fl = reinterpret_cast<const uint8_t *>(g.flags);
        for (int i = threadIdx.x; i < th * kWords; i += kThreads) {
            const int r = i >> 5, c = i & 31;
            if (c < nw) sflag[i] = fl[(((size_t)(y0 + r) * L + x0) >> 3) + c];
        }
    }
    __syncthreads();

    Counters cnt;

    // ---- colour 0 on rows -1..th (the tile and its ring rows), one warp per row
    for (int ry = warp - 1; ry <= th; ry += kWarps) {
        if (lane >= nw) continue;
        const int gy = wrap(y0 + ry, L);
        const uint32_t grp = (uint32_t)gy * (uint32_t)wpr + (uint32_t)(w0 + lane);
        const bool inside = ry >= 0 && ry < th;
        uint32_t fl = (kNE && inside) ? sflag[ry * kWords + lane] : 0u;
        uint2 nv;
        if ((gy & 1) == 0)
            nv = update<kNE, 0, false>(t, sthr, g, ry, lane, grp, ctr1, ctr2, 0u, fl, cnt);
        else
            nv = update<kNE, 1, false>(t, sthr, g, ry, lane, grp, ctr1, ctr2, 0u, fl, cnt);
        if (kNE && inside) sflag[ry * kWords + lane] = (uint8_t)fl;
        t.at(ry, lane) = nv;
    }
    // ---- colour 0 on the edge words: the site at column x0-1 is colour 0 on
    // odd rows (a parity-1 word at wx = -1), the one at x0+8*nw on even rows
    // (a parity-0 word at wx = nw).  Warp 0 takes odd rows, warp 1 even rows.
    if (warp < 2) {
        const int want = warp == 0 ? 1 : 0;
        for (int ry = lane; ry < th; ry += 32) {
            const int gy = y0 + ry;
            if ((gy & 1) != want) continue;
            const int gw = wrap(want ? w0 - 1 : w0 + nw, wpr);
            const uint32_t grp = (uint32_t)gy * (uint32_t)wpr + (uint32_t)gw;
            const int wx = want ? -1 : nw;
            uint32_t fl = 0;
            uint2 nv;
            if (want)
                nv = update<kNE, 1, false>(t, sthr, g, ry, wx, grp, ctr1, ctr2, 0u, fl, cnt);
            else
                nv = update<kNE, 0, false>(t, sthr, g, ry, wx, grp, ctr1, ctr2, 0u, fl, cnt);
            t.at(ry, wx) = nv;
        }
    }
    __syncthreads();

    // ---- colour 1 on the tile rows; results go to the other spin buffer
    for (int ry = warp; ry < th; ry += kWarps) {
        if (lane >= nw) continue;
        const int gy = y0 + ry;
        const uint32_t grp = (uint32_t)gy * (uint32_t)wpr + (uint32_t)(w0 + lane);
        uint32_t fl = kNE ? (uint32_t)sflag[ry * kWords + lane] : 0u;
        uint2 nv;
        if ((gy & 1) == 0)  // colour 1 on an even row sits at odd bytes
            nv = update<kNE, 1, true>(t, sthr, g, ry, lane, grp, ctr1, ctr2, 1u, fl, cnt);
        else
            nv = update<kNE, 0, true>(t, sthr, g, ry, lane, grp, ctr1, ctr2, 1u, fl, cnt);
        *reinterpret_cast<uint2 *>(dst + (size_t)gy * L + x0 + 8 * lane) = nv;
        if (kNE) reinterpret_cast<uint8_t *>(g.flags)[(((size_t)gy * L + x0) >> 3) + lane] = (uint8_t)fl;
    }

    // ---- per-sweep counters: warp reduce, then one atomic per CTA and counter
    const int rb = __reduce_add_sync(0xffffffffu, cnt.bond);
    const int rm = __reduce_add_sync(0xffffffffu, cnt.mag);
    const int ru = __reduce_add_sync(0xffffffffu, cnt.up);
    const int rf = kNE ? __reduce_add_sync(0xffffffffu, cnt.unfl) : 0;
    if (lane == 0) {
        red[warp][0] = rb;
        red[warp][1] = rm;
        red[warp][2] = ru;
        red[warp][3] = rf;
    }
    __syncthreads();
    if (threadIdx.x < (kNE ? 4 : 3)) {
        long long s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        add_counter(series_slot(g.ctrl, sweep) + threadIdx.x, s);
    }
}

}  // namespace

int default_tile_h() { return kDefTileH; }

bool tile_shape_ok(int tile_w, int tile_h)
{
    if (tile_w != 0 && tile_w != kTileW) return false;
    if (tile_h != 0 && (tile_h < 2 || tile_h > kMaxTileH)) return false;
    return true;
}

bool tiled_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && (g.L % 16) == 0)) return false;
    // Every non-always entry must have thr >= 1 (t' = thr - 1 >= 0).
    for (int k = 0; k < 16; ++k) {
        if ((k & 7) > 4) continue;
        if (!((g.always16 >> k) & 1u) && g.thr16[k] == 0u) return false;
    }
    return true;
}

cudaError_t launch_sweep_tiled(const Geom &g, int tile_w, int tile_h, int off, cudaStream_t st)
{
    (void)tile_w;
    TiledArgs a;
    a.g = g;
    a.tile_h = tile_h ? tile_h : kDefTileH;
    a.off = off;
    // Kernel-side table: t' = thr - 1, all ones = accept without a draw.
    for (int k = 0; k < 16; ++k)
        a.g.thr16[k] = ((g.always16 >> k) & 1u) ? 0xFFFFFFFFu : g.thr16[k] - 1u;
    const size_t smem = (size_t)(a.tile_h + 4) * kPitch * sizeof(uint2) + (size_t)a.tile_h * kWords;
    dim3 grid((unsigned)((g.L + kTileW - 1) / kTileW), (unsigned)((g.L + a.tile_h - 1) / a.tile_h));
    if (g.model == LAT_NE) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_sweep_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep_tiled<true><<<grid, kThreads, smem, st>>>(a);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_sweep_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep_tiled<false><<<grid, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lat
