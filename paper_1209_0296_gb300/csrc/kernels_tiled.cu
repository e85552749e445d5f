// kernels_tiled.cu -- one launch per sweep for 2D spin-1/2 lattices (Ising
// and North-East), int8 spins of +-1 in the checkerboard-planar layout,
// L a multiple of 32.
//
// The paper's GPU sweep (§III.A steps 5-8, Fig. 2) copies each sub-lattice
// with its boundary into shared memory, updates the red+blue sites, ends the
// kernel as a device-wide barrier, and relaunches for green+white: two
// launches and two passes over memory per sweep.  Here one launch does the
// whole sweep: each CTA stages a tile of 256 columns x tile_h rows of both
// colour planes plus a two-row / one-word halo in shared memory, updates
// colour 0 on the tile AND on the one-site ring around it (recomputing the
// ring is legal because every draw is keyed by site group and sweep, so the
// ring holds bit for bit what the neighbouring tile computes), then updates
// colour 1 on the tile.  Results go to the other spin buffer: one read and
// one write per site per sweep (plus the halo).
//
// Work item = one 4-byte word of a colour plane row = four same-colour
// sites = one Philox call.  A warp owns one tile row (32 words), so the row
// parity p is warp-uniform.  In the planar layout the north/south and
// same-column neighbours of the four sites are the other plane's words at
// the same index, and the row-shifted neighbours are that word funnel-
// shifted by one byte.  Bytes are 0x01 (+1) or 0xFF (-1), so bits 1..7 of a
// byte all equal "spin down": the number of down neighbours of four sites
// at once comes from a bit-sliced adder, and a scaled table index is
// assembled with masks only.  The acceptance table is held as t' = thr - 1
// (all ones = accept without a draw), so a move is accepted iff u <= t';
// lattices whose table has a never-accept entry (thr = 0, possible only for
// dE/T > 22) use the generic kernel.  For North-East the Philox call is
// skipped when none of the sites needs a draw (locked sites need none).
#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kTileCols = 256;      // lattice columns per tile
constexpr int kWords = 32;          // 4-byte words per plane row per tile
constexpr int kPitch = kWords + 8;  // smem words per plane row: 3 pad, halo, 32, halo, 3 pad
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxTileH = 64;
constexpr int kDefTileH = 64;

struct TiledArgs {
    Geom g;
    int tile_h;
    int off;  // sweep offset relative to ctrl->sweep
};

// Byte permute in PTX's generic mode, where bit 3 of a selector nibble
// replicates the sign bit of the selected byte over the output byte.
LAT_D uint32_t prmt_sign(uint32_t a, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(a), "r"(sel));
    return r;
}

struct Tile {
    uint32_t *w;  // [2 planes][tile_h + 4 rows][kPitch]
    int plane_words;
    LAT_D uint32_t &at(int c, int ry, int wx) const
    {
        return w[c * plane_words + (ry + 2) * kPitch + wx + 4];
    }
};

// Everything about one work item that does not need its random numbers.
struct Item {
    uint32_t S, U, D, Lf, R;  // site bytes and their north, south, west, east neighbours
    uint32_t t0, t1, t2, t3;  // acceptance thresholds t' (all ones = no draw needed)
    uint32_t locked;          // North-East: 0xFF bytes at locked sites
    bool need;
};

// Gather the four colour-C sites of plane word (ry, wx) whose row has parity
// P, count their down neighbours and look up their thresholds.
template <bool kNE, int C, int P>
LAT_D void prepare(const Tile &t, const uint32_t *sthr, int ry, int wx, Item &it)
{
    it.S = t.at(C, ry, wx);
    const uint32_t O = t.at(1 - C, ry, wx);
    it.U = t.at(1 - C, ry - 1, wx);  // north, row y-1
    it.D = t.at(1 - C, ry + 1, wx);  // south, row y+1
    if (P == 0) {  // x = 2j: left neighbour is j-1 of the other plane, right is j
        it.Lf = __funnelshift_l(t.at(1 - C, ry, wx - 1), O, 8);
        it.R = O;
    } else {       // x = 2j+1: left is j, right is j+1
        it.Lf = O;
        it.R = __funnelshift_r(O, t.at(1 - C, ry, wx + 1), 8);
    }
    const uint32_t U = it.U, D = it.D, Lf = it.Lf, R = it.R;
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
                         (it.S & 0x20202020u);
    const char *tb = reinterpret_cast<const char *>(sthr);
    it.t0 = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
    it.t1 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
    it.t2 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
    it.t3 = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
    it.locked = 0;
    if (kNE) {
        // §III.B: a site may change only if north (U) and east (R) are up.
        // Sign-replicating each byte of (U | R) gives an all-ones mask for a
        // locked site: it then needs no draw, and its flip is masked off.
        it.locked = U | R;
        it.t0 |= prmt_sign(it.locked, 0x8888u);
        it.t1 |= prmt_sign(it.locked, 0x9999u);
        it.t2 |= prmt_sign(it.locked, 0xAAAAu);
        it.t3 |= prmt_sign(it.locked, 0xBBBBu);
    }
    it.need = (it.t0 & it.t1 & it.t2 & it.t3) != 0xFFFFFFFFu;
}

// Accept/reject the four sites with their draws u; return the new word.
template <bool kNE>
LAT_D uint32_t finish(const Item &it, const U4 &u, uint32_t &changed)
{
    const uint32_t acc = (u.x <= it.t0 ? 1u : 0u) | (u.y <= it.t1 ? 2u : 0u) |
                         (u.z <= it.t2 ? 4u : 0u) | (u.w <= it.t3 ? 8u : 0u);
    // Byte mask 0xFE at each flipped site: +1 (0x01) <-> -1 (0xFF).
    uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu;
    if (kNE) {
        F &= ~it.locked;
        changed = ((((F >> 1) & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
    }
    return it.S ^ F;
}

LAT_D int wrap(int v, int n)
{
    v += (v < 0) ? n : 0;
    v -= (v >= n) ? n : 0;
    return v;
}

// Sum of the four bytes of x (each sum fits 16 bits).
LAT_D int byte_sum(uint32_t x)
{
    const uint32_t s = (x & 0x00FF00FFu) + ((x >> 8) & 0x00FF00FFu);
    return (int)((s & 0xFFFFu) + (s >> 16));
}

// Process the colour-C items of rows ry and ry + kWarps (the second only if
// `two`) at word `lane`: both rows have the same parity, so one warp-uniform
// branch serves both and their Philox chains interleave.
template <bool kNE, int C, int P>
LAT_D void do_pair(const Tile &t, const uint32_t *sthr, const PhiloxPre &pp, int ry, bool two,
                   bool active, int lane, uint32_t grp_a, uint32_t grp_b, uint32_t &nva,
                   uint32_t &nvb, Item &a, Item &b, uint32_t &cha, uint32_t &chb)
{
    prepare<kNE, C, P>(t, sthr, ry, lane, a);
    if (two) prepare<kNE, C, P>(t, sthr, ry + kWarps, lane, b);
    else b.need = false;
    const bool need = active && (a.need || b.need);
    // An item that needs no draw has t' = all ones at every site, so any u
    // accepts exactly as "no draw" would: a North-East warp skips Philox only
    // when no lane needs it, and otherwise every lane takes the (unused)
    // draws; Ising always draws (an item needing none is rare).
    U4 ua = U4{0u, 0u, 0u, 0u}, ub = ua;
    if (!kNE || __any_sync(0xffffffffu, need)) {
        ua = philox_item(pp, grp_a, (uint32_t)C);
        if (two) ub = philox_item(pp, grp_b, (uint32_t)C);
    }
    nva = finish<kNE>(a, ua, cha);
    if (two) nvb = finish<kNE>(b, ub, chb);
}

// One sweep of the tile (bx, by) of lattice g (by the whole CTA).  sthr: the
// lattice's 16-entry t' table in shared memory.  smem_raw: the tile buffer,
// sized for tile_h; red: [kWarps][4] ints.  Called by every thread.
template <bool kNE>
LAT_D void sweep_tile(const SweepView g, const uint32_t *sthr, int bx, int by, int tile_h, int off,
                      unsigned char *smem_raw, int (*red)[5])
{
    const int L = g.L;
    const int half = L >> 1;            // sites per plane row
    const int wpr = L >> 3;             // words per plane row (= Philox groups per row)
    const int x0 = bx * kTileCols;
    const int y0 = by * tile_h;
    const int nw = min(kWords, (L - x0) >> 3);
    const int th = min(tile_h, L - y0);
    const int w0 = x0 >> 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool active = lane < nw;

    Tile t;
    t.w = reinterpret_cast<uint32_t *>(smem_raw);
    t.plane_words = (tile_h + 4) * kPitch;
    uint8_t *sflag0 = smem_raw + (size_t)2 * t.plane_words * 4;  // [tile_h][32], colour-0 flags

    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const int8_t *src = (sweep & 1) ? g.s1 : g.s0;
    int8_t *dst = (sweep & 1) ? g.s0 : g.s1;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);

    // ---- stage both planes, rows y0-2 .. y0+th+1: 16-byte interior loads + halo words
    const int rows = th + 4;
    const int n16 = nw >> 2;  // 16-byte chunks per plane row
    for (int i = threadIdx.x; i < 2 * rows * 8; i += kThreads) {
        const int c = i / (rows * 8);
        const int rem = i - c * rows * 8;
        const int r = rem >> 3, k = rem & 7;
        if (k >= n16) continue;
        const int gy = wrap(y0 + r - 2, L);
        const uint4 v = *reinterpret_cast<const uint4 *>(src + (size_t)c * g.plane +
                                                         (size_t)gy * half + 4 * (w0 + 4 * k));
        *reinterpret_cast<uint4 *>(&t.at(c, r - 2, 4 * k)) = v;
    }
    for (int i = threadIdx.x; i < 2 * rows * 2; i += kThreads) {
        const int c = i / (rows * 2);
        const int rem = i - c * rows * 2;
        const int r = rem >> 1, side = rem & 1;
        const int gy = wrap(y0 + r - 2, L);
        const int gw = wrap(side ? w0 + nw : w0 - 1, wpr);
        t.at(c, r - 2, side ? nw : -1) = *reinterpret_cast<const uint32_t *>(
            src + (size_t)c * g.plane + (size_t)gy * half + 4 * (size_t)gw);
    }
    __syncthreads();

    const size_t row_bytes = (size_t)half;
    Item ia, ib;
    uint32_t cha = 0, chb = 0, nva = 0, nvb = 0;

    // ---- colour 0 on rows -1..th (the tile and its ring rows); warp w takes
    // rows w-1 and w-1+8, then w-1+16 and w-1+24, ...
    for (int ry = warp - 1; ry <= th; ry += 2 * kWarps) {
        const bool two = ry + kWarps <= th;
        const int gy = wrap(y0 + ry, L);
        const int gyb = wrap(y0 + ry + kWarps, L);
        const uint32_t ga = (uint32_t)gy * (uint32_t)wpr + (uint32_t)(w0 + lane);
        const uint32_t gb = (uint32_t)gyb * (uint32_t)wpr + (uint32_t)(w0 + lane);
        if ((gy & 1) == 0)
            do_pair<kNE, 0, 0>(t, sthr, pp, ry, two, active, lane, ga, gb, nva, nvb, ia, ib, cha, chb);
        else
            do_pair<kNE, 0, 1>(t, sthr, pp, ry, two, active, lane, ga, gb, nva, nvb, ia, ib, cha, chb);
        if (active) {
            t.at(0, ry, lane) = nva;
            if (two) t.at(0, ry + kWarps, lane) = nvb;
            if (ry >= 0 && ry < th) {
                *reinterpret_cast<uint32_t *>(dst + (size_t)gy * row_bytes + 4 * (size_t)(w0 + lane)) = nva;
                if (kNE) {
                    uint8_t *fp = g.flags + (size_t)gy * wpr + w0 + lane;
                    const uint8_t f = (uint8_t)(*fp | cha);
                    *fp = f;
                    sflag0[ry * kWords + lane] = f;
                }
            }
            const int ryb = ry + kWarps;
            if (two && ryb < th) {
                *reinterpret_cast<uint32_t *>(dst + (size_t)gyb * row_bytes + 4 * (size_t)(w0 + lane)) = nvb;
                if (kNE) {
                    uint8_t *fp = g.flags + (size_t)gyb * wpr + w0 + lane;
                    const uint8_t f = (uint8_t)(*fp | chb);
                    *fp = f;
                    sflag0[ryb * kWords + lane] = f;
                }
            }
        }
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
            if (want) prepare<kNE, 0, 1>(t, sthr, ry, wx, ia);
            else prepare<kNE, 0, 0>(t, sthr, ry, wx, ia);
            const U4 u = (!kNE || ia.need) ? philox_item(pp, grp, 0u) : U4{0u, 0u, 0u, 0u};
            t.at(0, ry, wx) = finish<kNE>(ia, u, cha);
        }
    }
    __syncthreads();

    // ---- colour 1 on the tile rows, with the sweep's counters.  Byte-wise
    // accumulators: ue counts 2 per unequal bond around a colour-1 site, dn
    // counts 2 per down spin; they are summed once at the end.
    const uint32_t M1 = 0x02020202u;
    uint32_t ue = 0, dn = 0, dr = 0;   // dr: 2 per site differing from the reference
    int items = 0, unfl = 0;
    const bool has_ref = g.ref != nullptr;
    for (int ry = warp; ry < th; ry += 2 * kWarps) {
        const bool two = ry + kWarps < th;
        const int gy = y0 + ry, gyb = y0 + ry + kWarps;
        const uint32_t ga = (uint32_t)gy * (uint32_t)wpr + (uint32_t)(w0 + lane);
        const uint32_t gb = (uint32_t)gyb * (uint32_t)wpr + (uint32_t)(w0 + lane);
        if ((gy & 1) == 0)  // colour 1 on an even row sits at odd columns
            do_pair<kNE, 1, 1>(t, sthr, pp, ry, two, active, lane, ga, gb, nva, nvb, ia, ib, cha, chb);
        else
            do_pair<kNE, 1, 0>(t, sthr, pp, ry, two, active, lane, ga, gb, nva, nvb, ia, ib, cha, chb);
        if (active) {
            *reinterpret_cast<uint32_t *>(dst + g.plane + (size_t)gy * row_bytes + 4 * (size_t)(w0 + lane)) = nva;
            ue += ((ia.U ^ nva) & M1) + ((ia.D ^ nva) & M1) + ((ia.Lf ^ nva) & M1) + ((ia.R ^ nva) & M1);
            dn += (nva & M1) + (t.at(0, ry, lane) & M1);
            if (has_ref) {
                const size_t o = (size_t)gy * row_bytes + 4 * (size_t)(w0 + lane);
                dr += ((nva ^ *reinterpret_cast<const uint32_t *>(g.ref + g.plane + o)) & M1) +
                      ((t.at(0, ry, lane) ^ *reinterpret_cast<const uint32_t *>(g.ref + o)) & M1);
            }
            ++items;
            if (kNE) {
                uint8_t *fp = g.flags + (size_t)g.rows * wpr + (size_t)gy * wpr + w0 + lane;
                const uint32_t f1 = *fp | cha;
                *fp = (uint8_t)f1;
                unfl += 8 - __popc(f1) - __popc((uint32_t)sflag0[ry * kWords + lane]);
            }
            if (two) {
                *reinterpret_cast<uint32_t *>(dst + g.plane + (size_t)gyb * row_bytes + 4 * (size_t)(w0 + lane)) = nvb;
                ue += ((ib.U ^ nvb) & M1) + ((ib.D ^ nvb) & M1) + ((ib.Lf ^ nvb) & M1) + ((ib.R ^ nvb) & M1);
                dn += (nvb & M1) + (t.at(0, ry + kWarps, lane) & M1);
                if (has_ref) {
                    const size_t o = (size_t)gyb * row_bytes + 4 * (size_t)(w0 + lane);
                    dr += ((nvb ^ *reinterpret_cast<const uint32_t *>(g.ref + g.plane + o)) & M1) +
                          ((t.at(0, ry + kWarps, lane) ^ *reinterpret_cast<const uint32_t *>(g.ref + o)) & M1);
                }
                ++items;
                if (kNE) {
                    uint8_t *fp = g.flags + (size_t)g.rows * wpr + (size_t)gyb * wpr + w0 + lane;
                    const uint32_t f1 = *fp | chb;
                    *fp = (uint8_t)f1;
                    unfl += 8 - __popc(f1) - __popc((uint32_t)sflag0[(ry + kWarps) * kWords + lane]);
                }
            }
        }
    }
    // bond over 4 colour-1 sites = 16 - 2 * (# unequal bonds); mag and up
    // over the 8 sites of the two plane words.
    const int d2 = byte_sum(dn);
    const int bond = 16 * items - byte_sum(ue);
    const int mag = 8 * items - d2;
    const int up = 8 * items - (d2 >> 1);
    const int acf = 8 * items - byte_sum(dr);   // overlap with the reference, both planes

    // ---- per-sweep counters: warp reduce, then one atomic per CTA and counter
    const int rb = __reduce_add_sync(0xffffffffu, bond);
    const int rm = __reduce_add_sync(0xffffffffu, mag);
    const int ru = __reduce_add_sync(0xffffffffu, up);
    const int rf = kNE ? __reduce_add_sync(0xffffffffu, unfl) : 0;
    const int ra = has_ref ? __reduce_add_sync(0xffffffffu, acf) : 0;
    if (lane == 0) {
        red[warp][0] = rb;
        red[warp][1] = rm;
        red[warp][2] = ru;
        red[warp][3] = rf;
        red[warp][4] = ra;
    }
    __syncthreads();
    if (threadIdx.x < (kNE ? 4 : 3)) {
        long long s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        add_counter(series_slot(g.ctrl, sweep) + threadIdx.x, s);
    } else if (has_ref && threadIdx.x == 4) {
        long long s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += red[w][4];
        add_counter(acf_slot(g.ctrl, sweep), s);
    }
}

size_t tile_smem_bytes(int tile_h) { return (size_t)2 * (tile_h + 4) * kPitch * 4 + (size_t)tile_h * kWords; }

template <bool kNE>
__global__ void __launch_bounds__(kThreads) k_sweep_tiled(TiledArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t sthr[16];
    __shared__ int red[kWarps][5];
    if (threadIdx.x < 16) sthr[threadIdx.x] = a.g.thr16[threadIdx.x];
    sweep_tile<kNE>(sweep_view(a.g), sthr, blockIdx.x, blockIdx.y, a.tile_h, a.off, smem_raw, red);
}

// Batched sweep: a persistent grid works through a list of (lattice, tile)
// items of many lattices of one model, one sweep each, taking items from a
// shared counter.  Each lattice keeps its own parameters, table, seed and
// sweep counter (its Geom in device memory), so every tile computes exactly
// what its lattice's own launch would.  Tiles of one lattice are
// independent within a sweep (they read one buffer and write the other).
// The descriptor is staged through shared memory into a register copy, so
// the tile's own shared-memory stores cannot alias it.
template <bool kNE>
__global__ void __launch_bounds__(kThreads) k_batch_tiled(const Geom *geoms, const uint2 *items,
                                                         int n_items, unsigned *next_item, int tile_h,
                                                         int off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Geom sg;
    __shared__ uint32_t sthr[16];
    __shared__ int red[kWarps][5];
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
        if (threadIdx.x < 16) sthr[threadIdx.x] = sg.thr16[threadIdx.x];
        const SweepView g = sweep_view(sg);
        __syncthreads();
        const int tiles_x = (g.L + kTileCols - 1) / kTileCols;
        const int bx = (int)(w.y % (unsigned)tiles_x), by = (int)(w.y / (unsigned)tiles_x);
        sweep_tile<kNE>(g, sthr, bx, by, tile_h, off, smem_raw, red);
        __syncthreads();
    }
}

}  // namespace

int default_tile_h() { return kDefTileH; }

bool tile_shape_ok(int tile_w, int tile_h)
{
    if (tile_w != 0 && tile_w != kTileCols) return false;
    if (tile_h != 0 && (tile_h < 2 || tile_h > kMaxTileH)) return false;
    return true;
}

bool tiled_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && (g.L % 32) == 0)) return false;
    if (g.cpl != nullptr || g.model == LAT_POTTS) return false;   // per-bond couplings: generic and wide kernels only
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
    const size_t smem = tile_smem_bytes(a.tile_h);
    dim3 grid((unsigned)((g.L + kTileCols - 1) / kTileCols), (unsigned)((g.L + a.tile_h - 1) / a.tile_h));
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

// Kernel-side copy of a lattice's description for the batched kernel: the
// compact table in t' = thr - 1 form.
Geom tiled_geom(const Geom &g)
{
    Geom k = g;
    for (int i = 0; i < 16; ++i)
        k.thr16[i] = ((g.always16 >> i) & 1u) ? 0xFFFFFFFFu : g.thr16[i] - 1u;
    return k;
}

int tiles_of(const Geom &g, int tile_h)
{
    const int th = tile_h ? tile_h : kDefTileH;
    return ((g.L + kTileCols - 1) / kTileCols) * ((g.L + th - 1) / th);
}

cudaError_t launch_batch_tiled(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int tile_h, int off, int grid, bool ne, cudaStream_t st)
{
    const int th = tile_h ? tile_h : kDefTileH;
    const size_t smem = tile_smem_bytes(th);  // <= 48 kB for tile_h <= 64
    if (ne)
        k_batch_tiled<true><<<grid, kThreads, smem, st>>>(geoms, items, n_items, next_item, th, off);
    else
        k_batch_tiled<false><<<grid, kThreads, smem, st>>>(geoms, items, n_items, next_item, th, off);
    return cudaGetLastError();
}

int batch_tiled_grid(bool ne)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ne)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_tiled<true>, kThreads, tile_smem_bytes(kDefTileH));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_tiled<false>, kThreads, tile_smem_bytes(kDefTileH));
    if (per < 1) per = 1;
    return sms * per;
}

}  // namespace lat
