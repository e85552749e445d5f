// kernels_tiled.cu -- one launch per sweep for 2D spin-1/2 lattices (Ising
// and North-East), int8 spins of +-1, L a multiple of 16.
//
// The paper's GPU sweep (§III.A steps 5-8, Fig. 2) copies each sub-lattice
// with its boundary into shared memory, updates the red+blue sites, ends the
// kernel as a device-wide barrier, and relaunches for green+white: two
// launches and two passes over memory per sweep.  Here one launch does the
// whole sweep: each CTA stages a tile plus a two-site halo in shared
// memory, updates colour 0 on the tile AND on a one-site ring around it
// (recomputing the ring is legal because every draw is keyed by site group
// and sweep, so the ring holds bit for bit what the neighbouring tile
// computes), then updates colour 1 on the tile and writes it straight back.
// HBM traffic is one read and one write per site per sweep.
//
// Each thread item is one 8-byte word of a row: four sites of the active
// colour (bytes p, p+2, p+4, p+6 with p = (colour + y) & 1), which is also
// one Philox call (4 same-colour sites per draw).  The neighbour counts of
// the four sites are formed with byte permutes and a bit-sliced adder over
// the down-flag bits (bytes are 0x01 for +1 and 0xFF for -1, so bits 1..7
// of a byte all equal "spin down").  The Philox call is skipped when none
// of the four sites needs a draw (dE <= 0 everywhere, or, for North-East,
// no site unlocked).
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kTiledThreads = 256;
constexpr int kMaxTileW = 512;   // columns (bytes)
constexpr int kMaxTileH = 64;    // rows
constexpr int kDefTileW = 256;
constexpr int kDefTileH = 32;

struct TiledArgs {
    Geom g;              // includes the compact table thr16 / always16
    int tile_w, tile_h;  // columns (multiple of 16), rows
    int off;             // sweep offset relative to ctrl->sweep
};

LAT_D uint32_t bperm(uint32_t a, uint32_t b, uint32_t sel) { return __byte_perm(a, b, sel); }

// Shared-memory tile: rows -2..tile_h+1, words -1..tile_w/8 (8 bytes each).
struct Smem {
    int pitch;  // words per row
    uint2 *w;   // [(tile_h+4) * pitch]
    LAT_D uint2 &at(int ry, int wx) const { return w[(ry + 2) * pitch + (wx + 1)]; }
};

struct Counters {
    int bond = 0, mag = 0, up = 0, unfl = 0;
};

// Update the four colour-`colour` sites of word (ry, wx).  Returns the
// 4-bit accept mask (bit q: site at byte p+2q flipped) and writes the new
// word through *out.  When `measure` is set (colour-1 pass) the counters
// of the word's final state are accumulated.
template <bool kNE>
LAT_D uint32_t update_word(const TiledArgs &a, const Smem &sm, const uint32_t *sthr, int ry, int wx,
                           uint32_t gy, uint32_t gw, int colour, unsigned long long sweep,
                           uint2 *out, bool measure, uint32_t flagbyte, Counters &cnt)
{
    const uint2 W = sm.at(ry, wx);
    const uint2 Wu = sm.at(ry - 1, wx);
    const uint2 Wd = sm.at(ry + 1, wx);
    const uint32_t wl_hi = sm.at(ry, wx - 1).y;
    const uint32_t wr_lo = sm.at(ry, wx + 1).x;

    const int p = (colour + (int)gy) & 1;
    const uint32_t sel = p ? 0x7531u : 0x6420u;  // bytes p, p+2, p+4, p+6 -> 0..3

    // Left neighbours: the word shifted up by one byte (byte b <- byte b-1).
    const uint32_t xl_lo = __funnelshift_l(wl_hi, W.x, 8);
    const uint32_t xl_hi = __funnelshift_l(W.x, W.y, 8);
    // Right neighbours: shifted down by one byte (byte b <- byte b+1).
    const uint32_t xr_lo = __funnelshift_r(W.x, W.y, 8);
    const uint32_t xr_hi = __funnelshift_r(W.y, wr_lo, 8);

    const uint32_t S = bperm(W.x, W.y, sel);
    const uint32_t U = bperm(Wu.x, Wu.y, sel);   // north: row y-1
    const uint32_t D = bperm(Wd.x, Wd.y, sel);   // south: row y+1
    const uint32_t Lf = bperm(xl_lo, xl_hi, sel);
    const uint32_t R = bperm(xr_lo, xr_hi, sel);  // east: column x+1

    // Bit-sliced count of down neighbours (0..4) per byte, valid in bits 1..7.
    const uint32_t s1 = U ^ D ^ Lf;
    const uint32_t c1 = (U & D) | (U & Lf) | (D & Lf);
    const uint32_t b0 = s1 ^ R;
    const uint32_t c2 = s1 & R;
    const uint32_t b1 = c1 ^ c2;
    const uint32_t b2 = c1 & c2;
    // 4-bit table index per byte: sd << 3 | nd.
    const uint32_t idx = ((b0 >> 1) & 0x01010101u) | (b1 & 0x02020202u) | ((b2 << 1) & 0x04040404u) |
                         ((S << 2) & 0x08080808u);
    // North-East: unlocked iff north and east are up (bit 1 clear in both).
    const uint32_t unlocked = kNE ? ~(U | R) : 0xFFFFFFFFu;

    uint32_t need = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t iq = (idx >> (8 * q)) & 0xFu;
        const uint32_t ok = (unlocked >> (8 * q + 1)) & 1u;
        need |= (ok & ~(a.g.always16 >> iq) & 1u) << q;
    }
    uint32_t acc = 0;
    if (need != 0) {
        const uint32_t g = gy * a.g.G + gw;
        const U4 u = philox(U4{g, (uint32_t)sweep, (uint32_t)(sweep >> 32), (uint32_t)colour},
                            a.g.key0, a.g.key1);
        const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t iq = (idx >> (8 * q)) & 0xFu;
            const uint32_t ok = (unlocked >> (8 * q + 1)) & 1u;
            const uint32_t hit = ((a.g.always16 >> iq) & 1u) | (uw[q] < sthr[iq] ? 1u : 0u);
            acc |= (hit & ok) << q;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t iq = (idx >> (8 * q)) & 0xFu;
            const uint32_t ok = (unlocked >> (8 * q + 1)) & 1u;
            acc |= (((a.g.always16 >> iq) & 1u) & ok) << q;
        }
    }
    // Flip accepted sites: +1 (0x01) <-> -1 (0xFF) is an XOR with 0xFE.
    const uint32_t F = ((acc & 1u) ? 0x000000FEu : 0u) | ((acc & 2u) ? 0x0000FE00u : 0u) |
                       ((acc & 4u) ? 0x00FE0000u : 0u) | ((acc & 8u) ? 0xFE000000u : 0u);
    uint2 Wn;
    if (p) {
        Wn.x = W.x ^ bperm(F, 0u, 0x1404u);
        Wn.y = W.y ^ bperm(F, 0u, 0x3424u);
    } else {
        Wn.x = W.x ^ bperm(F, 0u, 0x4140u);
        Wn.y = W.y ^ bperm(F, 0u, 0x4342u);
    }
    *out = Wn;

    if (measure) {
        // Bond sum over this word's colour-1 sites: s' * (sum of the four
        // colour-0 neighbours) = 2 * (# equal neighbours) - 4 per site.
        const uint32_t Sn = S ^ F;
        const uint32_t M1 = 0x02020202u;
        const int eq = __popc(~(Sn ^ U) & M1) + __popc(~(Sn ^ D) & M1) + __popc(~(Sn ^ Lf) & M1) +
                       __popc(~(Sn ^ R) & M1);
        cnt.bond += 2 * eq - 16;
        const int downs = __popc(Wn.x & M1) + __popc(Wn.y & M1);
        cnt.mag += 8 - 2 * downs;
        cnt.up += 8 - downs;
        if (kNE) {
            const uint32_t fb = flagbyte | (((acc & 1u) | ((acc & 2u) << 1) | ((acc & 4u) << 2) |
                                             ((acc & 8u) << 3)) << p);
            cnt.unfl += 8 - __popc(fb);
        }
    }
    return acc;
}

template <bool kNE>
__global__ void __launch_bounds__(kTiledThreads) k_sweep_tiled(TiledArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t sthr[16];
    __shared__ long long red[kTiledThreads / 32];

    const Geom &g = a.g;
    const int L = g.L;
    const uint32_t words_per_row = (uint32_t)L >> 3;  // = G (4 sites of one colour per word)
    const int x0 = blockIdx.x * a.tile_w;
    const int y0 = blockIdx.y * a.tile_h;
    const int tw = min(a.tile_w, L - x0);
    const int th = min(a.tile_h, L - y0);
    const int nw = tw >> 3;  // words per tile row
    const uint32_t w0 = (uint32_t)x0 >> 3;

    Smem sm;
    sm.pitch = (a.tile_w >> 3) + 2;
    sm.w = reinterpret_cast<uint2 *>(smem_raw);
    uint8_t *sflag = smem_raw + (size_t)(a.tile_h + 4) * sm.pitch * sizeof(uint2);  // [tile_h][nw]

    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)a.off;
    const int8_t *src = g.s[sweep & 1];
    int8_t *dst = g.s[(sweep + 1) & 1];

    // Stage rows y0-2 .. y0+th+1, words w0-1 .. w0+nw (periodic wrap).
    const int rows_ld = th + 4, cols_ld = nw + 2;
    for (int t = threadIdx.x; t < rows_ld * cols_ld; t += blockDim.x) {
        const int ry = t / cols_ld - 2;
        const int wx = t % cols_ld - 1;
        const uint32_t gy = (uint32_t)((y0 + ry + L) % L);
        const uint32_t gw = (w0 + (uint32_t)wx + words_per_row) % words_per_row;
        sm.at(ry, wx) = *reinterpret_cast<const uint2 *>(src + (size_t)gy * L + (size_t)gw * 8);
    }
    if (kNE) {
        const uint8_t *fl = reinterpret_cast<const uint8_t *>(g.flags);
        for (int t = threadIdx.x; t < th * nw; t += blockDim.x) {
            const int ry = t / nw, wx = t % nw;
            sflag[ry * nw + wx] = fl[((size_t)(y0 + ry) * L + x0) / 8 + wx];
        }
    }
    __syncthreads();

    Counters cnt;

    // Colour 0 on rows -1..th (tile plus ring rows) ...
    const int n0 = (th + 2) * nw;
    // ... plus, per tile row, the one edge word whose colour-0 site touches the tile.
    for (int t = threadIdx.x; t < n0 + th; t += blockDim.x) {
        int ry, wx;
        if (t < n0) {
            ry = t / nw - 1;
            wx = t % nw;
        } else {
            ry = t - n0;
            const uint32_t gyr = (uint32_t)(y0 + ry);
            wx = (gyr & 1u) ? -1 : nw;  // x0-1 is colour 0 on odd rows, x0+tw on even rows
        }
        const uint32_t gy = (uint32_t)((y0 + ry + L) % L);
        const uint32_t gw = (w0 + (uint32_t)wx + words_per_row) % words_per_row;
        uint2 nwv;
        const uint32_t acc = update_word<kNE>(a, sm, sthr, ry, wx, gy, gw, 0, sweep, &nwv, false, 0u, cnt);
        sm.at(ry, wx) = nwv;
        if (kNE && acc != 0 && ry >= 0 && ry < th && wx >= 0 && wx < nw) {
            const int p = (int)(gy & 1u);
            sflag[ry * nw + wx] |= (uint8_t)((((acc & 1u) | ((acc & 2u) << 1) | ((acc & 4u) << 2) |
                                                ((acc & 8u) << 3))) << p);
        }
    }
    __syncthreads();

    // Colour 1 on the tile; results go straight to global memory.
    for (int t = threadIdx.x; t < th * nw; t += blockDim.x) {
        const int ry = t / nw, wx = t % nw;
        const uint32_t gy = (uint32_t)(y0 + ry);
        const uint32_t gw = w0 + (uint32_t)wx;
        uint2 nwv;
        const uint32_t fb = kNE ? (uint32_t)sflag[ry * nw + wx] : 0u;
        const uint32_t acc = update_word<kNE>(a, sm, sthr, ry, wx, gy, gw, 1, sweep, &nwv, true, fb, cnt);
        *reinterpret_cast<uint2 *>(dst + (size_t)gy * L + (size_t)gw * 8) = nwv;
        if (kNE) {
            const int p = (int)((1u + gy) & 1u);
            const uint32_t nb = fb | ((((acc & 1u) | ((acc & 2u) << 1) | ((acc & 4u) << 2) |
                                        ((acc & 8u) << 3))) << p);
            reinterpret_cast<uint8_t *>(g.flags)[((size_t)gy * L + x0) / 8 + wx] = (uint8_t)nb;
        }
    }

    unsigned long long *slot = series_slot(g.ctrl, sweep);
    long long v;
    v = block_sum_ll(cnt.bond, red);
    if (threadIdx.x == 0) add_counter(slot + 0, v);
    v = block_sum_ll(cnt.mag, red);
    if (threadIdx.x == 0) add_counter(slot + 1, v);
    v = block_sum_ll(cnt.up, red);
    if (threadIdx.x == 0) add_counter(slot + 2, v);
    if (kNE) {
        v = block_sum_ll(cnt.unfl, red);
        if (threadIdx.x == 0) add_counter(slot + 3, v);
    }
}

}  // namespace

bool tile_shape_ok(int tile_w, int tile_h)
{
    if (tile_w != 0 && (tile_w < 16 || tile_w > kMaxTileW || (tile_w & 15))) return false;
    if (tile_h != 0 && (tile_h < 2 || tile_h > kMaxTileH)) return false;
    return true;
}

bool tiled_supported(const Geom &g)
{
    return g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && (g.L % 16) == 0;
}

cudaError_t launch_sweep_tiled(const Geom &g, int tile_w, int tile_h, int off, cudaStream_t st)
{
    TiledArgs a;
    a.g = g;
    a.tile_w = tile_w ? tile_w : kDefTileW;
    a.tile_h = tile_h ? tile_h : kDefTileH;
    a.off = off;
    const int pitch = (a.tile_w >> 3) + 2;
    const size_t smem = (size_t)(a.tile_h + 4) * pitch * sizeof(uint2) + (size_t)a.tile_h * (a.tile_w >> 3);
    dim3 grid((unsigned)((g.L + a.tile_w - 1) / a.tile_w), (unsigned)((g.L + a.tile_h - 1) / a.tile_h));
    if (g.model == LAT_NE) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_sweep_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep_tiled<true><<<grid, kTiledThreads, smem, st>>>(a);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_sweep_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep_tiled<false><<<grid, kTiledThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lat
