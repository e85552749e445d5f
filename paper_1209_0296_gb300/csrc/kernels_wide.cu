// kernels_wide.cu -- two launches per sweep (one per colour, the kernel
// boundary being the device-wide barrier of §III.A steps 6-7) for 2D
// spin-1/2 lattices (Ising and North-East), int8 spins of +-1 in the
// checkerboard-planar layout, L a multiple of 32.
//
// A thread owns 16 consecutive same-colour sites of one plane row (one
// 16-byte load = four Philox groups), so the loads, index arithmetic and
// Philox set-up are shared by 16 sites.  The colour-c sites only read the
// other plane, so the colour-c pass never reads a byte another thread
// writes: colour 0 reads buffer s[sweep & 1] and writes the new colour-0
// sites plus a copy of the colour-1 sites into s[(sweep+1) & 1]; colour 1
// then updates s[(sweep+1) & 1] in place and reduces the sweep's counters.
// Neighbour counts, thresholds and acceptance are those of the tiled kernel
// (bytes 0x01 / 0xFF, bit-sliced adder, t' = thr - 1 table).
//
// Uniform Ising lattices run k_wide_pipe: each thread walks one chunk
// column down the rows with two chunks in flight, so the Philox draws of
// one chunk (wide multiplies) and the Metropolis step of the other (logic)
// share each instruction block.  North-East lattices and lattices with
// per-site disorder run k_wide_half_* (one chunk at a time, grid-stride).
#include <algorithm>

#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;

// Byte permute in PTX's generic mode, where bit 3 of a selector nibble
// replicates the sign bit of the selected byte over the output byte.
LAT_D uint32_t prmt_sign(uint32_t a, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(a), "r"(sel));
    return r;
}

LAT_D int byte_sum(uint32_t x)
{
    const uint32_t s = (x & 0x00FF00FFu) + ((x >> 8) & 0x00FF00FFu);
    return (int)((s & 0xFFFFu) + (s >> 16));
}

struct Counts {
    int bond = 0, mag = 0, up = 0, unfl = 0, acf = 0, fld = 0;
};

// W consecutive 4-byte words (4W same-colour sites) from p.
template <int W>
LAT_D void load_words(const int8_t *p, uint32_t (&v)[W])
{
    if constexpr (W == 4) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else if constexpr (W == 2) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
        v[0] = *reinterpret_cast<const uint32_t *>(p);
    }
}

template <int W>
LAT_D void store_words(int8_t *p, const uint32_t (&v)[W])
{
    if constexpr (W == 4) *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
    else if constexpr (W == 2) *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
    else *reinterpret_cast<uint32_t *>(p) = v[0];
}

// Sweep colour `colour` of the chunk k (4W sites, W Philox groups) of plane
// row y.  The two-launch kernel uses W = 4 (16 sites, one 16-byte load per
// row); the resident kernel uses smaller W on small lattices, for more
// threads with shorter dependency chains.  kInPlace: both buffers are the
// same array (the resident kernel), so colour 0 does not copy the colour-1
// sites.  kCpl: per-site disorder bytes (Eq. 1 couplings); kFld (with
// kCpl): also per-site field signs, whose -h entries are table entries
// 16..31, and the field sum sum_i eta_i s_i.
template <bool kNE, bool kInPlace = false, int W = 4, bool kPre = false, bool kCpl = false, bool kFld = false>
LAT_D void wide_chunk(const SweepView g, const uint32_t *sthr, int colour, unsigned long long sweep,
                      const PhiloxPre &pp, int y, int k, Counts &cnt, const U4 *upre = nullptr)
{
    const int8_t *src = (sweep & 1) ? g.s1 : g.s0;
    int8_t *dst = (sweep & 1) ? g.s0 : g.s1;
    if (colour == 1) src = dst;
    const int L = g.L;
    const uint32_t half = g.half;
    const int oc = 1 - colour;
    const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
    const uint32_t nwr = half >> 2;  // 4-byte words per plane row
    auto row = [&](int c, int r) { return src + (uint64_t)c * g.plane + (uint64_t)r * half; };
    uint32_t S[W], O[W], U[W], D[W];
    load_words<W>(row(colour, y) + 4 * W * k, S);
    load_words<W>(row(oc, y) + 4 * W * k, O);
    load_words<W>(row(oc, ym) + 4 * W * k, U);   // north
    load_words<W>(row(oc, yp) + 4 * W * k, D);   // south
    const bool p1 = ((colour + y) & 1) != 0;
    uint32_t adj;
    {
        const uint32_t w = p1 ? (uint32_t)(W * k + W) : (uint32_t)(W * k - 1 + nwr);
        adj = reinterpret_cast<const uint32_t *>(row(oc, y))[wrap_once(w, nwr)];
    }
    // Ising in the two-launch kernels: the draws do not depend on the loaded
    // words, so they are made while the loads are in flight (a North-East
    // item may skip them: its locked sites need none).
    constexpr bool kEarly = !kNE && !kPre && !kInPlace;
    U4 u[W];
#pragma unroll
    for (int w = 0; w < W; ++w) u[w] = U4{0, 0, 0, 0};
    if constexpr (kEarly) {
        const uint32_t g0 = (uint32_t)y * g.G + (uint32_t)(W * k);
#pragma unroll
        for (int w = 0; w < W; ++w) u[w] = philox_item(pp, g0 + (uint32_t)w, (uint32_t)colour);
    }
    uint32_t Lf[W], R[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        if (!p1) {  // x = 2j: west is j-1 of the other plane, east is j
            Lf[w] = __funnelshift_l(w == 0 ? adj : O[w - 1], O[w], 8);
            R[w] = O[w];
        } else {    // x = 2j+1: west is j, east is j+1
            Lf[w] = O[w];
            R[w] = __funnelshift_r(O[w], w == W - 1 ? adj : O[w + 1], 8);
        }
    }
    uint32_t C[W];   // disorder bytes of the colour-c sites (kCpl)
    if constexpr (kCpl) {
        // Eq. 1 couplings: a negative bond enters the energy as a flipped
        // neighbour, so XOR 0xFE (+1 <-> -1) into that neighbour's byte
        load_words<W>(reinterpret_cast<const int8_t *>(g.cpl) + (uint64_t)colour * g.plane + (uint64_t)y * half +
                          4 * W * k, C);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            Lf[w] ^= ((C[w] >> 0) & 0x01010101u) * 0xFEu;
            R[w] ^= ((C[w] >> 1) & 0x01010101u) * 0xFEu;
            U[w] ^= ((C[w] >> 2) & 0x01010101u) * 0xFEu;
            D[w] ^= ((C[w] >> 3) & 0x01010101u) * 0xFEu;
        }
    }
    uint32_t t[W][4], locked[W];
    bool need = false;
    const char *tb = reinterpret_cast<const char *>(sthr);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t s1 = U[w] ^ D[w] ^ Lf[w];
        const uint32_t c1 = (U[w] & D[w]) | (U[w] & Lf[w]) | (D[w] & Lf[w]);
        const uint32_t b0 = s1 ^ R[w];
        const uint32_t b1 = c1 ^ (s1 & R[w]);
        const uint32_t b2 = c1 & s1 & R[w];
        // byte offset into the 16-entry table (index sd<<3 | nd, 4 bytes each)
        uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) | (S[w] & 0x20202020u);
        if constexpr (kFld) idx |= C[w] & 0x40404040u;   // eta_i = -1: the -h entries 16..31
        t[w][0] = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
        t[w][1] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
        t[w][2] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
        t[w][3] = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
        locked[w] = 0;
        if constexpr (kNE) {
            // §III.B: north (U) and east (R) must be up; a locked site needs
            // no draw (t' all ones) and its flip is masked off below.
            locked[w] = U[w] | R[w];
            t[w][0] |= prmt_sign(locked[w], 0x8888u);
            t[w][1] |= prmt_sign(locked[w], 0x9999u);
            t[w][2] |= prmt_sign(locked[w], 0xAAAAu);
            t[w][3] |= prmt_sign(locked[w], 0xBBBBu);
        }
        need |= (t[w][0] & t[w][1] & t[w][2] & t[w][3]) != 0xFFFFFFFFu;
    }
    // An item that needs no draw has t' = all ones at every site, so any u
    // accepts exactly as "no draw" would.
    if constexpr (kPre) {   // draws made by the caller (same groups, same counters)
#pragma unroll
        for (int w = 0; w < W; ++w) u[w] = upre[w];
    } else if (!kEarly && need) {
        const uint32_t g0 = (uint32_t)y * g.G + (uint32_t)(W * k);
#pragma unroll
        for (int w = 0; w < W; ++w) u[w] = philox_item(pp, g0 + (uint32_t)w, (uint32_t)colour);
    }
    uint32_t Sn[W], chg = 0;
    const uint32_t M1 = 0x02020202u;
    uint32_t ue = 0, dn = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t acc = (u[w].x <= t[w][0] ? 1u : 0u) | (u[w].y <= t[w][1] ? 2u : 0u) |
                             (u[w].z <= t[w][2] ? 4u : 0u) | (u[w].w <= t[w][3] ? 8u : 0u);
        uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu;  // 0xFE at flipped sites
        if constexpr (kNE) {
            F &= ~locked[w];
            chg |= ((((F >> 1) & 0x01010101u) * 0x01020408u) >> 24 & 0xFu) << (8 * w);
        }
        Sn[w] = S[w] ^ F;
        if (colour == 1) {
            // bond: 4 - 2 * (# unequal) per colour-1 site (2 per unequal bond below)
            ue += ((U[w] ^ Sn[w]) & M1) + ((D[w] ^ Sn[w]) & M1) + ((Lf[w] ^ Sn[w]) & M1) +
                  ((R[w] ^ Sn[w]) & M1);
            dn += (Sn[w] & M1) + (O[w] & M1);  // 2 per down spin, both planes
        }
    }
    store_words<W>(dst + (uint64_t)colour * g.plane + (uint64_t)y * half + 4 * W * k, Sn);
    if (colour == 0 && !kInPlace) store_words<W>(dst + (uint64_t)g.plane + (uint64_t)y * half + 4 * W * k, O);
    int unfl = 0;
    if constexpr (kNE) {
        // persistence bytes of the W groups (bit q = site 4m+q)
        uint8_t *fb = g.flags + ((uint64_t)colour * L + y) * g.G + (uint64_t)(W * k);
        const uint8_t *fob = g.flags + ((uint64_t)oc * L + y) * g.G + (uint64_t)(W * k);
        uint32_t f, fo = 0;
        if constexpr (W == 4) {
            uint32_t *fp = reinterpret_cast<uint32_t *>(fb);
            f = *fp | chg;
            *fp = f;
            if (colour == 1) fo = *reinterpret_cast<const uint32_t *>(fob);
        } else if constexpr (W == 2) {
            uint16_t *fp = reinterpret_cast<uint16_t *>(fb);
            f = (uint32_t)*fp | chg;
            *fp = (uint16_t)f;
            if (colour == 1) fo = *reinterpret_cast<const uint16_t *>(fob);
        } else {
            f = (uint32_t)*fb | chg;
            *fb = (uint8_t)f;
            if (colour == 1) fo = *fob;
        }
        if (colour == 1) unfl = 8 * W - __popc(f) - __popc(fo);
    }
    if (colour == 1) {
        const int d2 = byte_sum(dn);
        cnt.bond += 16 * W - byte_sum(ue);
        cnt.mag += 8 * W - d2;
        cnt.up += 8 * W - (d2 >> 1);
        cnt.unfl += unfl;
        if (g.ref != nullptr) {
            // overlap with the reference over both planes' 8W sites:
            // 8W - 2 * (# sites that differ); 0x02 marks a differing byte
            uint32_t R1[W], R0[W], dr = 0;
            load_words<W>(g.ref + g.plane + (uint64_t)y * half + 4 * W * k, R1);
            load_words<W>(g.ref + (uint64_t)y * half + 4 * W * k, R0);
#pragma unroll
            for (int w = 0; w < W; ++w) dr += ((Sn[w] ^ R1[w]) & M1) + ((O[w] ^ R0[w]) & M1);
            cnt.acf += 8 * W - byte_sum(dr);
        }
    }
    if constexpr (kFld) {
        // field sum over this colour's 4W sites (final after this launch:
        // each colour adds its own sites, so no launch reads the other
        // plane's disorder bytes); eta_i s_i is down when exactly one of
        // (s_i down: bit 1, eta_i = -1: bit 6) holds
        uint32_t ed = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) ed += (Sn[w] ^ (C[w] >> 5)) & M1;
        cnt.fld += 4 * W - byte_sum(ed);
    }
}

// Add the block's counters to the sweep's slot (bond, mag, up[, unflipped]).
// Warp sums go to shared memory and warp 0 adds them up.  32-bit partial
// sums are enough: a block's |bond| is at most 2 per site it updated, and a
// block never updates 2^30 sites in one call.
// acf: the sweep's autocorrelation slot, or null when no reference is set.
LAT_D void flush_slot(unsigned long long *slot, unsigned long long *acf, const Counts &c, bool ne,
                      int (*red)[5])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = __reduce_add_sync(0xffffffffu, c.bond);
    const int rm = __reduce_add_sync(0xffffffffu, c.mag);
    const int ru = __reduce_add_sync(0xffffffffu, c.up);
    const int rf = __reduce_add_sync(0xffffffffu, c.unfl);
    const int ra = acf ? __reduce_add_sync(0xffffffffu, c.acf) : 0;
    if (lane == 0) {
        red[warp][0] = rb;
        red[warp][1] = rm;
        red[warp][2] = ru;
        red[warp][3] = rf;
        red[warp][4] = ra;
    }
    __syncthreads();
    if (warp == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        const int b = __reduce_add_sync(0xffffffffu, in ? red[lane][0] : 0);
        const int m = __reduce_add_sync(0xffffffffu, in ? red[lane][1] : 0);
        const int u = __reduce_add_sync(0xffffffffu, in ? red[lane][2] : 0);
        const int f = __reduce_add_sync(0xffffffffu, in ? red[lane][3] : 0);
        if (lane < (ne ? 4 : 3)) add_counter(slot + lane, (long long)(lane == 0 ? b : lane == 1 ? m : lane == 2 ? u : f));
        if (acf) {
            const int a = __reduce_add_sync(0xffffffffu, in ? red[lane][4] : 0);
            if (lane == 0) add_counter(acf, (long long)a);
        }
    }
    __syncthreads();
}

LAT_D void flush(const SweepView &g, unsigned long long sweep, const Counts &c, bool ne, int (*red)[5])
{
    flush_slot(series_slot(g.ctrl, sweep), g.ref ? acf_slot(g.ctrl, sweep) : nullptr, c, ne, red);
}

// Add one int per thread, summed over the block, to *dst (all threads call).
LAT_D void flush_one(unsigned long long *dst, int v, int (*red)[5])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) red[warp][0] = r;
    __syncthreads();
    if (warp == 0) {
        const int t = __reduce_add_sync(0xffffffffu, lane < (int)(blockDim.x >> 5) ? red[lane][0] : 0);
        if (lane == 0) add_counter(dst, (long long)t);
    }
    __syncthreads();
}

// kFld: 32-entry table, entries 16..31 built from the -h half of the full
// table (t' = thr - 1 form, all ones = always), index sd << 3 | nd as for
// entries 0..15.
template <bool kNE, bool kCpl, bool kFld>
LAT_D void wide_half_body(const Geom &g, int colour, int off, uint32_t *sthr, int (*red)[5])
{
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    if constexpr (kFld) {
        if (threadIdx.x >= 16 && threadIdx.x < 32) {
            const int k = threadIdx.x - 16, nd = k & 7;
            uint32_t t = 0u;
            if (nd <= 4) {
                const int ds = (k >> 3) ? 2 : -2, n = 4 - 2 * nd;
                const TabEntry e = g.tab[(2 * g.dsmax + 1) * g.nn + (ds + g.dsmax) * g.nn + (n + g.nmax)];
                t = e.always ? 0xFFFFFFFFu : e.thr - 1u;
            }
            sthr[threadIdx.x] = t;
        }
    }
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const uint32_t cpr = g.half >> 4;  // 16-site chunks per plane row
    Counts cnt;
    const SweepView v = sweep_view(g);
    // Grid-stride over chunks with one resident wave of CTAs: the counter
    // reduction (and its barrier) happens once per CTA, not once per chunk.
    for (GridWalk w((uint32_t)g.L, cpr); w.ok(); w.next())
        wide_chunk<kNE, false, 4, false, kCpl, kFld>(v, sthr, colour, sweep, pp, (int)w.r, (int)w.k, cnt);
    if (colour == 1) flush(v, sweep, cnt, kNE, red);
    if constexpr (kFld) flush_one(fld_slot(g.ctrl, sweep), cnt.fld, red);   // both colours
}

// Per-bond couplings (Eq. 1, J_ij = J eps_ij), uniform field.
__global__ void __launch_bounds__(kThreads) k_wide_half_cpl(Geom g, int colour, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    wide_half_body<false, true, false>(g, colour, off, sthr, red);
}

// Couplings and field signs: bounded to three CTAs per SM (80 registers);
// unbounded it takes 120 and only two fit.
__global__ void __launch_bounds__(kThreads, 3) k_wide_half_fld(Geom g, int colour, int off)
{
    __shared__ uint32_t sthr[32];
    __shared__ int red[kThreads / 32][5];
    wide_half_body<false, true, true>(g, colour, off, sthr, red);
}

// North-East: bounded to three CTAs per SM (80 registers); unbounded it
// takes 117 and only two fit.
__global__ void __launch_bounds__(kThreads, 3) k_wide_half_ne(Geom g, int colour, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    wide_half_body<true, false, false>(g, colour, off, sthr, red);
}

// ---------------------------------------------------------------------
// Software-pipelined two-launch Ising sweep (uniform J and h, no per-site
// disorder).  Same chunks, draws, table and bits as wide_chunk<false>; the
// difference is the schedule.  A chunk costs two kinds of work that load
// different pipes: its four Philox4x32-10 calls (wide multiplies on the
// FMA pipe) and the Metropolis step (logic on the ALU pipe).  Done one
// after the other they keep one pipe idle while the other works, so each
// iteration here loads and draws chunk i+1 in the same straight-line block
// as the Metropolis step of chunk i, and the two streams interleave.
// ---------------------------------------------------------------------
struct WideIn {
    uint32_t S[4], O[4], U[4], D[4];
    uint32_t adj;
};

// What one thread needs to walk its chunk column k (16 sites) down the
// rows of one colour: the rows it visits are y0, y0 + rs, y0 + 2 rs, ...
// with rs * cpr threads in the grid, so the column, its row-end neighbour
// word and its base addresses are fixed and a row costs a few 32-bit adds.
template <int kColour>
struct ColWalk {
    const int8_t *pS;      // this colour's sites before the sweep, + 16k
    const int8_t *pO;      // the other colour's current sites, + 16k
    const int8_t *pOrow;   // the other colour's current sites (row starts)
    int8_t *dS;            // this colour's plane in the new buffer, + 16k
    const int8_t *r1, *r0; // reference planes 1 and 0, + 16k (or null)
    uint32_t half, L, G, k;
    uint32_t adjb0, adjb1; // byte offset in the row of the neighbour word past the chunk end, x parity 0 / 1
};

// old: the buffer of the state before the sweep; nw: the new buffer.
// Colour 0 reads both planes of old; colour 1 reads its own sites from old
// (colour 0 did not touch them) and the new colour-0 sites from nw.  Each
// colour writes only its own plane of nw, so no plane is copied.
template <int kColour>
LAT_D ColWalk<kColour> col_walk(const SweepView &g, const int8_t *old, int8_t *nw, uint32_t k)
{
    constexpr int oc = 1 - kColour;
    ColWalk<kColour> c;
    const uint32_t plane = (uint32_t)g.plane;   // N < 2^32, so a plane is < 2^31 bytes
    c.pOrow = (kColour == 0 ? old : nw) + (size_t)oc * plane;
    c.pS = old + (size_t)kColour * plane + 16 * k;
    c.pO = c.pOrow + 16 * k;
    c.dS = nw + (size_t)kColour * plane + 16 * k;
    c.r1 = g.ref ? g.ref + (size_t)plane + 16 * k : nullptr;
    c.r0 = g.ref ? g.ref + 16 * k : nullptr;
    c.half = g.half;
    c.L = (uint32_t)g.L;
    c.G = g.G;
    c.k = k;
    const uint32_t nwr = g.half >> 2;   // 4-byte words per plane row
    c.adjb0 = 4u * wrap_once(4u * k - 1u + nwr, nwr);   // x = 2j: west word before the chunk
    c.adjb1 = 4u * wrap_once(4u * k + 4u, nwr);         // x = 2j+1: east word after it
    return c;
}

// Loads of the walk's chunk in plane row y.
template <int kColour>
LAT_D void col_load(const ColWalk<kColour> &c, uint32_t y, WideIn &in)
{
    const uint32_t oy = y * c.half;
    const uint32_t oym = y == 0 ? oy + (c.L - 1) * c.half : oy - c.half;
    const uint32_t oyp = y == c.L - 1 ? 0u : oy + c.half;
    load_words<4>(c.pS + oy, in.S);
    load_words<4>(c.pO + oy, in.O);
    load_words<4>(c.pO + oym, in.U);   // north
    load_words<4>(c.pO + oyp, in.D);   // south
    in.adj = *reinterpret_cast<const uint32_t *>(c.pOrow + oy + (((kColour + y) & 1) ? c.adjb1 : c.adjb0));
}

// The four Philox groups of the walk's chunk in plane row y.
template <int kColour>
LAT_D void col_draws(const PhiloxPre &pp, const ColWalk<kColour> &c, uint32_t y, U4 (&u)[4])
{
    const uint32_t g0 = y * c.G + 4u * c.k;
#pragma unroll
    for (int w = 0; w < 4; ++w) u[w] = philox_item(pp, g0 + (uint32_t)w, (uint32_t)kColour);
}

// The Metropolis step of one loaded chunk: neighbour counts, table, accept
// iff u <= t', write; colour 1 also counts bonds, magnetisation and up
// sites (and the overlap with the reference when kRef).
template <int kColour, bool kRef>
LAT_D void col_step(const ColWalk<kColour> &c, const uint32_t *sthr, uint32_t y, const WideIn &in,
                    const U4 (&u)[4], Counts &cnt)
{
    const uint32_t oy = y * c.half;
    const bool p1 = ((kColour + y) & 1) != 0;
    const char *tb = reinterpret_cast<const char *>(sthr);
    const uint32_t M1 = 0x02020202u;
    uint32_t Sn[4], ue = 0, dn = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t Lf, R;
        if (!p1) {   // x = 2j: west is j-1 of the other plane, east is j
            Lf = __funnelshift_l(w == 0 ? in.adj : in.O[w - 1], in.O[w], 8);
            R = in.O[w];
        } else {     // x = 2j+1: west is j, east is j+1
            Lf = in.O[w];
            R = __funnelshift_r(in.O[w], w == 3 ? in.adj : in.O[w + 1], 8);
        }
        const uint32_t Uw = in.U[w], Dw = in.D[w];
        const uint32_t s1 = Uw ^ Dw ^ Lf;
        const uint32_t c1 = (Uw & Dw) | (Uw & Lf) | (Dw & Lf);
        const uint32_t b0 = s1 ^ R;
        const uint32_t b1 = c1 ^ (s1 & R);
        const uint32_t b2 = c1 & s1 & R;
        const uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) | (in.S[w] & 0x20202020u);
        const uint32_t t0 = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
        const uint32_t t1 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
        const uint32_t t2 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
        const uint32_t t3 = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
        const uint32_t acc = (u[w].x <= t0 ? 1u : 0u) | (u[w].y <= t1 ? 2u : 0u) | (u[w].z <= t2 ? 4u : 0u) |
                             (u[w].w <= t3 ? 8u : 0u);
        // (the spread multiplies run on the FMA pipe, which has room; the
        // logic pipe is the busier one)
        const uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu;   // 0xFE at flipped sites
        Sn[w] = in.S[w] ^ F;
        if constexpr (kColour == 1) {
            // unequal bonds, 2 per pair: the adder's sum and carry words
            // (U^D^Lf, maj(U,D,Lf)) against the new spin count the unequal
            // bonds to U, D, Lf once and twice (every bit of a byte above
            // bit 0 repeats the "down" flag), R counts once
            ue += ((s1 ^ Sn[w]) & M1) + ((c1 ^ Sn[w]) & 0x04040404u) + ((R ^ Sn[w]) & M1);
            dn += (Sn[w] & M1) + (in.O[w] & M1);
        }
    }
    store_words<4>(c.dS + oy, Sn);
    if constexpr (kColour == 1) {
        const int d2 = byte_sum(dn);
        cnt.bond += 64 - byte_sum(ue);
        cnt.mag += 32 - d2;
        cnt.up += 32 - (d2 >> 1);
        if constexpr (kRef) {
            uint32_t R1[4], R0[4], dr = 0;
            load_words<4>(c.r1 + oy, R1);
            load_words<4>(c.r0 + oy, R0);
#pragma unroll
            for (int w = 0; w < 4; ++w) dr += ((Sn[w] ^ R1[w]) & M1) + ((in.O[w] ^ R0[w]) & M1);
            cnt.acf += 32 - byte_sum(dr);
        }
    }
}

constexpr int kPipeMinB = 2;   // CTAs per SM (the two chunks in flight need ~100 registers)

template <int kColour, bool kRef>
__global__ void __launch_bounds__(kThreads, kPipeMinB) k_wide_pipe(Geom g, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const SweepView v = sweep_view(g);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    Counts cnt;
    // thread -> (chunk column k, first row y); rs rows between visits.  The
    // launch has at least cpr threads, and rs * cpr of them work.
    const uint32_t cpr = g.half >> 4;
    const uint32_t rs = (gridDim.x * blockDim.x) / cpr;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t y = gt / cpr;
    const uint32_t k = gt - y * cpr;
    if (y < rs && y < (uint32_t)g.L) {
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        const ColWalk<kColour> c = col_walk<kColour>(v, old, nw, k);
        const uint32_t L = (uint32_t)g.L;
        // Two chunks in flight, in registers A and B in turn: each block
        // loads and draws one chunk while the Metropolis step of the other
        // runs (no copies between the two).
        WideIn A, B;
        U4 uA[4], uB[4];
        col_load<kColour>(c, y, A);
        col_draws<kColour>(pp, c, y, uA);
        for (;;) {
            const uint32_t y1 = y + rs;
            if (y1 >= L) {
                col_step<kColour, kRef>(c, sthr, y, A, uA, cnt);
                break;
            }
            col_load<kColour>(c, y1, B);
            col_draws<kColour>(pp, c, y1, uB);
            col_step<kColour, kRef>(c, sthr, y, A, uA, cnt);
            const uint32_t y2 = y1 + rs;
            if (y2 >= L) {
                col_step<kColour, kRef>(c, sthr, y1, B, uB, cnt);
                break;
            }
            col_load<kColour>(c, y2, A);
            col_draws<kColour>(pp, c, y2, uA);
            col_step<kColour, kRef>(c, sthr, y1, B, uB, cnt);
            y = y2;
        }
    }
    if constexpr (kColour == 1) flush(v, sweep, cnt, false, red);
}

// ---------------------------------------------------------------------
// Any even L: one Philox group (the up to four same-colour sites
// j = 4m .. 4m+3 of a plane row) per thread and row.  A plane row holds
// L/2 bytes, so for L % 8 != 0 rows do not start on a word boundary and the
// last group of a row holds L/2 % 4 sites; a group's bytes are gathered
// from the aligned words that hold them, the neighbour past the group's
// edge (west of site 4m, or east of its last site, across the periodic
// row end when the group is the row's last) is one byte load, and a
// partial or misaligned group is written byte by byte (its neighbours'
// bytes belong to other threads).  The SWAR step is the wide kernel's on
// one word, with the bytes past the last site masked off.
// ---------------------------------------------------------------------

// The bytes p[0 .. nv) (1 <= nv <= 4) as one word, byte k = p[k], the
// bytes from nv on unspecified.  Read from the aligned words that hold
// them; the word after the last needed byte is not read, so every word
// read holds an in-bounds byte (and the spin buffers are multiples of 4
// bytes: N = L^2 with L even).
LAT_D uint32_t load_group(const int8_t *p, uint32_t nv)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t sh = (uint32_t)(a & 3u);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a - sh);
    const uint32_t lo = w[0];
    const uint32_t hi = (sh + nv > 4u) ? w[1] : 0u;
    return __funnelshift_r(lo, hi, 8u * sh);
}

LAT_D void store_group(int8_t *p, uint32_t v, uint32_t nv)
{
    if (nv == 4u && (reinterpret_cast<uintptr_t>(p) & 3u) == 0u) {
        *reinterpret_cast<uint32_t *>(p) = v;
    } else {
        for (uint32_t k = 0; k < nv; ++k) p[k] = (int8_t)(v >> (8u * k));
    }
}

struct GroupIn {
    uint32_t S, O, U, D;   // the group's sites, the other plane's same-index, north and south words
    uint32_t nb;           // the other plane's byte past the group's edge (west of 4m, or east of the last site)
};

// One thread's column of groups (group m of every plane row it visits).
template <int kColour>
struct GroupWalk {
    const int8_t *pS;      // this colour's sites before the sweep (plane base)
    const int8_t *pO;      // the other colour's current sites (plane base)
    int8_t *dS;            // this colour's plane in the new buffer
    const int8_t *r1, *r0; // reference planes 1 and 0 (or null)
    uint8_t *fc;           // persistence bytes of this colour, group m of row 0 (North-East)
    const uint8_t *fo;     // persistence bytes of the other colour, group m of row 0
    uint32_t half, L, G, m, j0, nv, vmask;
    uint32_t jprev, jnext; // row index of the west neighbour of site j0 / the east neighbour of the last site
};

template <int kColour>
LAT_D GroupWalk<kColour> group_walk(const SweepView &g, const int8_t *old, int8_t *nw, uint32_t m)
{
    constexpr int oc = 1 - kColour;
    GroupWalk<kColour> c;
    const uint32_t plane = (uint32_t)g.plane;
    c.pS = old + (size_t)kColour * plane;
    c.pO = (kColour == 0 ? old : nw) + (size_t)oc * plane;
    c.dS = nw + (size_t)kColour * plane;
    c.r1 = g.ref ? g.ref + (size_t)plane : nullptr;
    c.r0 = g.ref;
    c.fc = g.flags ? g.flags + (size_t)kColour * g.rows * g.G + m : nullptr;
    c.fo = g.flags ? g.flags + (size_t)oc * g.rows * g.G + m : nullptr;
    c.half = g.half;
    c.L = (uint32_t)g.L;
    c.G = g.G;
    c.m = m;
    c.j0 = 4u * m;
    c.nv = min(4u, g.half - c.j0);
    c.vmask = c.nv == 4u ? 0xFFFFFFFFu : (1u << (8u * c.nv)) - 1u;
    c.jprev = c.j0 == 0u ? g.half - 1u : c.j0 - 1u;
    c.jnext = c.j0 + c.nv == g.half ? 0u : c.j0 + c.nv;
    return c;
}

template <int kColour>
LAT_D void group_load(const GroupWalk<kColour> &c, uint32_t y, GroupIn &in)
{
    const uint32_t oy = y * c.half;
    const uint32_t oym = y == 0 ? oy + (c.L - 1) * c.half : oy - c.half;
    const uint32_t oyp = y == c.L - 1 ? 0u : oy + c.half;
    in.S = load_group(c.pS + oy + c.j0, c.nv);
    in.O = load_group(c.pO + oy + c.j0, c.nv);
    in.U = load_group(c.pO + oym + c.j0, c.nv);   // north
    in.D = load_group(c.pO + oyp + c.j0, c.nv);   // south
    in.nb = (uint32_t)(uint8_t)c.pO[oy + (((kColour + y) & 1) ? c.jnext : c.jprev)];
}

template <int kColour>
LAT_D U4 group_draw(const PhiloxPre &pp, const GroupWalk<kColour> &c, uint32_t y)
{
    return philox_item(pp, y * c.G + c.m, (uint32_t)kColour);
}

template <int kColour, bool kNE, bool kRef>
LAT_D void group_step(const GroupWalk<kColour> &c, const uint32_t *sthr, uint32_t y, const GroupIn &in, const U4 &u,
                      Counts &cnt)
{
    const uint32_t oy = y * c.half;
    const bool p1 = ((kColour + y) & 1) != 0;
    const char *tb = reinterpret_cast<const char *>(sthr);
    const uint32_t M1 = 0x02020202u;
    uint32_t Lf, R;
    if (!p1) {   // x = 2j: west is j-1 of the other plane (nb for site j0), east is j
        Lf = (in.O << 8) | in.nb;
        R = in.O;
    } else {     // x = 2j+1: west is j, east is j+1 (nb for the last site)
        Lf = in.O;
        R = ((in.O >> 8) & (c.vmask >> 8)) | (in.nb << (8u * (c.nv - 1u)));
    }
    const uint32_t s1 = in.U ^ in.D ^ Lf;
    const uint32_t c1 = (in.U & in.D) | (in.U & Lf) | (in.D & Lf);
    const uint32_t b0 = s1 ^ R;
    const uint32_t b1 = c1 ^ (s1 & R);
    const uint32_t b2 = c1 & s1 & R;
    const uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) | (in.S & 0x20202020u);
    uint32_t t0 = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
    uint32_t t1 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
    uint32_t t2 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
    uint32_t t3 = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
    uint32_t locked = 0;
    if constexpr (kNE) {   // §III.B: north (U) and east (R) must be up
        locked = in.U | R;
        t0 |= prmt_sign(locked, 0x8888u);
        t1 |= prmt_sign(locked, 0x9999u);
        t2 |= prmt_sign(locked, 0xAAAAu);
        t3 |= prmt_sign(locked, 0xBBBBu);
    }
    const uint32_t acc = (u.x <= t0 ? 1u : 0u) | (u.y <= t1 ? 2u : 0u) | (u.z <= t2 ? 4u : 0u) | (u.w <= t3 ? 8u : 0u);
    uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu & c.vmask;   // 0xFE at flipped sites
    if constexpr (kNE) F &= ~locked;
    const uint32_t Sn = in.S ^ F;
    store_group(c.dS + oy + c.j0, Sn, c.nv);
    uint32_t fl = 0;
    if constexpr (kNE) {
        const uint32_t chg = (((F >> 1) & 0x01010101u) * 0x01020408u) >> 24 & 0xFu;
        uint8_t *fp = c.fc + (size_t)y * c.G;
        fl = (uint32_t)*fp | chg;
        *fp = (uint8_t)fl;
    }
    if constexpr (kColour == 1) {
        const uint32_t ue = (((s1 ^ Sn) & M1) + ((c1 ^ Sn) & 0x04040404u) + ((R ^ Sn) & M1)) & c.vmask;
        const uint32_t dn = ((Sn & M1) + (in.O & M1)) & c.vmask;
        const int d2 = byte_sum(dn);
        const int nv = (int)c.nv;
        cnt.bond += 4 * nv - byte_sum(ue);
        cnt.mag += 2 * nv - d2;
        cnt.up += 2 * nv - (d2 >> 1);
        if constexpr (kNE) cnt.unfl += 2 * nv - __popc(fl) - __popc((uint32_t)c.fo[(size_t)y * c.G]);
        if constexpr (kRef) {
            const uint32_t R1 = load_group(c.r1 + oy + c.j0, c.nv), R0 = load_group(c.r0 + oy + c.j0, c.nv);
            const uint32_t dr = (((Sn ^ R1) & M1) + ((in.O ^ R0) & M1)) & c.vmask;
            cnt.acf += 2 * nv - byte_sum(dr);
        }
    }
}

template <int kColour, bool kNE, bool kRef>
__global__ void __launch_bounds__(kThreads, 3) k_group_pipe(Geom g, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const SweepView v = sweep_view(g);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    Counts cnt;
    // thread -> (group m, first row y); rs rows between visits (the launch
    // has at least G threads, rs * G of them work)
    const uint32_t G = g.G;
    const uint32_t rs = (gridDim.x * blockDim.x) / G;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t y = gt / G;
    const uint32_t m = gt - y * G;
    if (y < rs && y < (uint32_t)g.L) {
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        const GroupWalk<kColour> c = group_walk<kColour>(v, old, nw, m);
        const uint32_t L = (uint32_t)g.L;
        // two groups in flight (A and B in turn), as in k_wide_pipe
        GroupIn A, B;
        U4 uA, uB;
        group_load<kColour>(c, y, A);
        uA = group_draw<kColour>(pp, c, y);
        for (;;) {
            const uint32_t y1 = y + rs;
            if (y1 >= L) {
                group_step<kColour, kNE, kRef>(c, sthr, y, A, uA, cnt);
                break;
            }
            group_load<kColour>(c, y1, B);
            uB = group_draw<kColour>(pp, c, y1);
            group_step<kColour, kNE, kRef>(c, sthr, y, A, uA, cnt);
            const uint32_t y2 = y1 + rs;
            if (y2 >= L) {
                group_step<kColour, kNE, kRef>(c, sthr, y1, B, uB, cnt);
                break;
            }
            group_load<kColour>(c, y2, A);
            uA = group_draw<kColour>(pp, c, y2);
            group_step<kColour, kNE, kRef>(c, sthr, y1, B, uB, cnt);
            y = y2;
        }
    }
    if constexpr (kColour == 1) flush(v, sweep, cnt, kNE, red);
}

// Batched form of the any-L kernel: items are (lattice, band of rows) of
// one colour; the CTA's threads take the band's groups in row-major order.
constexpr uint32_t kGroupItemGroups = 2048;   // about 8 groups per thread per item

LAT_HD uint32_t group_band_rows(uint32_t G) { return G >= kGroupItemGroups ? 1u : kGroupItemGroups / G; }

template <int kColour, bool kNE>
LAT_D void batch_group_item(const SweepView &v, const uint32_t *sthr, uint32_t band, Counts &cnt)
{
    const unsigned long long sweep = v.ctrl->sweep;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), v.key0, v.key1);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    const uint32_t G = v.G, L = (uint32_t)v.L;
    const uint32_t br = group_band_rows(G);
    const uint32_t y0 = band * br;
    const uint32_t y1 = min(L, y0 + br);
    const uint32_t total = (y1 - y0) * G;
    // walk t = tid, tid + 256, ... over the band as (row, group), without a
    // division per step
    uint32_t t = threadIdx.x;
    uint32_t r = t / G, m = t - r * G;
    const uint32_t sr = kThreads / G, sm = kThreads - sr * G;
    for (; t < total; t += kThreads) {
        const GroupWalk<kColour> c = group_walk<kColour>(v, old, nw, m);
        GroupIn in;
        group_load<kColour>(c, y0 + r, in);
        const U4 u = group_draw<kColour>(pp, c, y0 + r);
        if (v.ref != nullptr) group_step<kColour, kNE, true>(c, sthr, y0 + r, in, u, cnt);
        else group_step<kColour, kNE, false>(c, sthr, y0 + r, in, u, cnt);
        r += sr;
        m += sm;
        if (m >= G) {
            m -= G;
            ++r;
        }
    }
}

template <bool kNE>
__global__ void __launch_bounds__(kThreads, 3) k_batch_group(const Geom *geoms, const uint2 *items, int n_items,
                                                           unsigned *next_item, int colour)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    __shared__ Geom sg;
    __shared__ int cur;
    int loaded = -1;
    for (;;) {
        if (threadIdx.x == 0) cur = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int it = cur;
        if (it >= n_items) break;
        const uint2 w = items[it];
        if ((int)w.x != loaded) {
            if (threadIdx.x < sizeof(Geom) / 4)
                reinterpret_cast<uint32_t *>(&sg)[threadIdx.x] =
                    reinterpret_cast<const uint32_t *>(&geoms[w.x])[threadIdx.x];
            __syncthreads();
            if (threadIdx.x < 16) sthr[threadIdx.x] = sg.thr16[threadIdx.x];
            loaded = (int)w.x;
            __syncthreads();
        }
        const SweepView v = sweep_view(sg);
        Counts cnt;
        if (colour == 0) {
            batch_group_item<0, kNE>(v, sthr, w.y, cnt);
        } else {
            batch_group_item<1, kNE>(v, sthr, w.y, cnt);
            flush(v, v.ctrl->sweep, cnt, kNE, red);   // ends with __syncthreads()
        }
        __syncthreads();
    }
}

// Batched form: a persistent grid takes (lattice, item) pairs from an
// atomic counter; an item is kItemChunks x kThreads chunks of one colour of
// one lattice.  The descriptor and table are reloaded only when a CTA moves
// to another lattice (items are ordered by lattice); the sweep works on a
// register copy of the descriptor.
constexpr int kItemChunks = 4;

template <bool kNE>
__global__ void __launch_bounds__(kThreads, kNE ? 2 : 3) k_batch_wide(const Geom *geoms, const uint2 *items, int n_items,
                                                        unsigned *next_item, int colour)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    __shared__ Geom sg;
    __shared__ int cur;
    int loaded = -1;
    for (;;) {
        if (threadIdx.x == 0) cur = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int it = cur;
        if (it >= n_items) break;
        const uint2 w = items[it];
        if ((int)w.x != loaded) {
            if (threadIdx.x < sizeof(Geom) / 4)
                reinterpret_cast<uint32_t *>(&sg)[threadIdx.x] =
                    reinterpret_cast<const uint32_t *>(&geoms[w.x])[threadIdx.x];
            __syncthreads();
            if (threadIdx.x < 16) sthr[threadIdx.x] = sg.thr16[threadIdx.x];
            loaded = (int)w.x;
            __syncthreads();
        }
        const SweepView v = sweep_view(sg);
        const unsigned long long sweep = v.ctrl->sweep;
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), v.key0, v.key1);
        const uint32_t cpr = v.half >> 4;
        const uint32_t total = (uint32_t)v.L * cpr;
        Counts cnt;
#pragma unroll 1
        for (int c = 0; c < kItemChunks; ++c) {
            const uint32_t t = (w.y * (uint32_t)kItemChunks + (uint32_t)c) * kThreads + threadIdx.x;
            if (t >= total) break;
            wide_chunk<kNE>(v, sthr, colour, sweep, pp, (int)(t / cpr), (int)(t % cpr), cnt);
        }
        if (colour == 1) flush(v, sweep, cnt, kNE, red);   // ends with __syncthreads()
        __syncthreads();
    }
}

// Resident form for lattices that fit in one CTA's shared memory (§III.A
// with the whole lattice as the block's tile): the CTA loads the spins (and
// the North-East persistence bytes) once, runs n sweeps in place -- an
// in-place checkerboard update is exact because a colour reads only the
// other colour, and __syncthreads() is the barrier between the two -- and
// writes the final state to s[(sweep + n) & 1].  One launch replaces 2n.
constexpr int kResThreads = 512;
constexpr size_t kResMaxBytes = 220 * 1024;

// One lattice, n_sweeps sweeps, by the whole CTA.  g may live in shared
// memory (the batched kernel): the sweep loop reads only register copies.
// advance: the CTA also moves the lattice's sweep counter on by n_sweeps.
template <bool kNE, int W>
LAT_D void resident_body(const Geom &g, int off, int n_sweeps, bool advance, uint4 *res_smem, uint32_t *sthr,
                         int (*red)[5])
{
    int8_t *sp = reinterpret_cast<int8_t *>(res_smem);
    const uint64_t n16 = g.N >> 4;                       // N % 16 == 0 (L % 32 == 0)
    const uint64_t f16 = kNE ? ((uint64_t)2 * g.rows * g.G) >> 4 : 0;  // flag bytes / 16
    uint4 *fl4 = res_smem + n16;
    const unsigned long long sweep0 = g.ctrl->sweep + (unsigned long long)off;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(g.s[sweep0 & 1]);
        for (uint64_t i = threadIdx.x; i < n16; i += blockDim.x) res_smem[i] = src[i];
        if constexpr (kNE) {
            const uint4 *fsrc = reinterpret_cast<const uint4 *>(g.flags);
            for (uint64_t i = threadIdx.x; i < f16; i += blockDim.x) fl4[i] = fsrc[i];
        }
    }
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    SweepView v = sweep_view(g);
    v.s0 = sp;
    v.s1 = sp;
    v.flags = reinterpret_cast<uint8_t *>(fl4);
    const uint32_t cpr = g.half / (4 * W);
    const uint32_t total = (uint32_t)g.L * cpr;
    unsigned long long *slot0 = series_slot(g.ctrl, sweep0);  // slots of consecutive sweeps are contiguous
    unsigned long long *acf0 = g.ref ? acf_slot(g.ctrl, sweep0) : nullptr;
    // With at most one chunk per thread and colour, a thread draws both
    // colours' numbers at the start of the sweep: the colour-1 draws do not
    // depend on the colour-0 result, so their Philox chain leaves the
    // critical path.
    const bool one = W == 1 && total <= blockDim.x;   // (register budget: narrow chunks only)
    const int y1 = (int)(threadIdx.x / cpr), k1 = (int)(threadIdx.x % cpr);
    for (int s = 0; s < n_sweeps; ++s) {
        const unsigned long long sweep = sweep0 + (unsigned long long)s;
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        Counts cnt;
        if (W == 1 && one) {
            const bool act = threadIdx.x < total;
            U4 u0[W], u1[W];
            if (act) {
                const uint32_t g0 = (uint32_t)y1 * g.G + (uint32_t)(W * k1);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    u0[w] = philox_item(pp, g0 + (uint32_t)w, 0u);
                    u1[w] = philox_item(pp, g0 + (uint32_t)w, 1u);
                }
                wide_chunk<kNE, true, W, true>(v, sthr, 0, sweep, pp, y1, k1, cnt, u0);
            }
            __syncthreads();
            if (act) wide_chunk<kNE, true, W, true>(v, sthr, 1, sweep, pp, y1, k1, cnt, u1);
        } else {
            for (uint32_t t = threadIdx.x; t < total; t += blockDim.x)
                wide_chunk<kNE, true, W>(v, sthr, 0, sweep, pp, (int)(t / cpr), (int)(t % cpr), cnt);
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < total; t += blockDim.x)
                wide_chunk<kNE, true, W>(v, sthr, 1, sweep, pp, (int)(t / cpr), (int)(t % cpr), cnt);
        }
        flush_slot(slot0 + 4ull * (unsigned)s, acf0 ? acf0 + (unsigned)s : nullptr, cnt, kNE, red);  // ends with __syncthreads()
    }
    {
        uint4 *dst = reinterpret_cast<uint4 *>(g.s[(sweep0 + (unsigned long long)n_sweeps) & 1]);
        for (uint64_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = res_smem[i];
        if constexpr (kNE) {
            uint4 *fdst = reinterpret_cast<uint4 *>(g.flags);
            for (uint64_t i = threadIdx.x; i < f16; i += blockDim.x) fdst[i] = fl4[i];
        }
    }
    if (advance) {
        __syncthreads();   // every thread has read the old counter long before
        if (threadIdx.x == 0) g.ctrl->sweep = sweep0 + (unsigned long long)n_sweeps;
    }
}

template <bool kNE, int W>
__global__ void __launch_bounds__(kResThreads, 1) k_resident(Geom g, int off, int n_sweeps)
{
    extern __shared__ uint4 res_smem[];
    __shared__ uint32_t sthr[16];
    __shared__ int red[kResThreads / 32][5];
    resident_body<kNE, W>(g, off, n_sweeps, false, res_smem, sthr, red);
}

// Batched form: CTA i sweeps lattice i (descriptor geoms[i]) by
// min(chunk, n[i] - done) sweeps and advances its counter; lattices of
// either model and width share the launch.
__global__ void __launch_bounds__(kResThreads, 1) k_batch_resident(const Geom *geoms, const long long *n,
                                                                   long long done, int chunk)
{
    extern __shared__ uint4 res_smem[];
    __shared__ uint32_t sthr[16];
    __shared__ int red[kResThreads / 32][5];
    __shared__ Geom sg;
    const long long left = n[blockIdx.x] - done;
    if (left <= 0) return;   // uniform over the CTA
    const int m = (int)(left < (long long)chunk ? left : (long long)chunk);
    if (threadIdx.x < sizeof(Geom) / 4)
        reinterpret_cast<uint32_t *>(&sg)[threadIdx.x] = reinterpret_cast<const uint32_t *>(&geoms[blockIdx.x])[threadIdx.x];
    __syncthreads();
    const bool narrow = (uint64_t)sg.L * (sg.half >> 2) <= (uint64_t)kResThreads;
    if (sg.model == LAT_NE) {
        if (narrow) resident_body<true, 1>(sg, 0, m, true, res_smem, sthr, red);
        else resident_body<true, 4>(sg, 0, m, true, res_smem, sthr, red);
    } else {
        if (narrow) resident_body<false, 1>(sg, 0, m, true, res_smem, sthr, red);
        else resident_body<false, 4>(sg, 0, m, true, res_smem, sthr, red);
    }
}

size_t resident_bytes(const Geom &g)
{
    return (size_t)g.N + (g.model == LAT_NE ? (size_t)2 * g.rows * g.G : 0);
}

}  // namespace

bool wide_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && (g.L % 32) == 0)) return false;
    if (g.model == LAT_POTTS) return false;
    for (int k = 0; k < 16; ++k) {
        if ((k & 7) > 4) continue;
        if (!((g.always16 >> k) & 1u) && g.thr16[k] == 0u) return false;
    }
    return true;
}

int wide_chunks(const Geom &g) { return (int)(((uint64_t)g.L * (g.half >> 4) + kThreads - 1) / kThreads); }

bool group_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && g.cpl == nullptr && (g.L % 2) == 0)) return false;
    if (g.model == LAT_POTTS) return false;
    for (int k = 0; k < 16; ++k) {
        if ((k & 7) > 4) continue;
        if (!((g.always16 >> k) & 1u) && g.thr16[k] == 0u) return false;
    }
    return true;
}

int group_items(const Geom &g)
{
    const uint32_t br = group_band_rows(g.G);
    return (int)(((uint32_t)g.L + br - 1) / br);
}

int batch_group_grid(bool ne)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ne) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_group<true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_group<false>, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_group(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item, int colour,
                               bool ne, int grid, cudaStream_t st)
{
    if (ne) k_batch_group<true><<<grid, kThreads, 0, st>>>(geoms, items, n_items, next_item, colour);
    else k_batch_group<false><<<grid, kThreads, 0, st>>>(geoms, items, n_items, next_item, colour);
    return cudaGetLastError();
}

cudaError_t launch_sweep_wide(const Geom &g, bool fields, int off, cudaStream_t st)
{
    const Geom k = tiled_geom(g);  // compact table in t' = thr - 1 form
    int dev = 0;
    cudaGetDevice(&dev);
    // one wave: SMs x resident CTAs per SM, queried once per kernel
    auto wave = [dev](const void *fn, int &cache) {
        if (cache == 0) {
            int sms = 0, per = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, 0);
            cache = sms * (per > 0 ? per : 1);
        }
        return cache;
    };
    if (!wide_supported(g)) {   // L % 32 != 0: the any-L group kernels
        static int res_group = 0;
        const uint64_t groups = (uint64_t)g.L * g.G;
        const unsigned gb = (unsigned)std::min<long long>(
            (long long)((groups + kThreads - 1) / kThreads),
            wave(reinterpret_cast<const void *>(k_group_pipe<1, true, true>), res_group));
        using KG = void (*)(Geom, int);
        const bool ne = g.model == LAT_NE, ref = k.ref != nullptr;
        const KG c0 = ne ? (ref ? k_group_pipe<0, true, true> : k_group_pipe<0, true, false>)
                         : (ref ? k_group_pipe<0, false, true> : k_group_pipe<0, false, false>);
        const KG c1 = ne ? (ref ? k_group_pipe<1, true, true> : k_group_pipe<1, true, false>)
                         : (ref ? k_group_pipe<1, false, true> : k_group_pipe<1, false, false>);
        c0<<<gb, kThreads, 0, st>>>(k, off);
        c1<<<gb, kThreads, 0, st>>>(k, off);
        return cudaGetLastError();
    }
    if (g.model != LAT_NE && g.cpl == nullptr) {   // uniform Ising: the software-pipelined kernels
        static int res_pipe = 0;
        const unsigned pb = (unsigned)std::min<long long>(
            wide_chunks(g), wave(reinterpret_cast<const void *>(k_wide_pipe<1, true>), res_pipe));
        if (k.ref != nullptr) {
            k_wide_pipe<0, true><<<pb, kThreads, 0, st>>>(k, off);
            k_wide_pipe<1, true><<<pb, kThreads, 0, st>>>(k, off);
        } else {
            k_wide_pipe<0, false><<<pb, kThreads, 0, st>>>(k, off);
            k_wide_pipe<1, false><<<pb, kThreads, 0, st>>>(k, off);
        }
        return cudaGetLastError();
    }
    // North-East, Ising with per-bond couplings, Ising with couplings and
    // per-site field signs
    const int m = g.model == LAT_NE ? 0 : (fields ? 2 : 1);
    using K = void (*)(Geom, int, int);
    const K kern[3] = {k_wide_half_ne, k_wide_half_cpl, k_wide_half_fld};
    static int resident[3] = {0, 0, 0};
    const unsigned blocks = (unsigned)std::min<long long>(
        wide_chunks(g), wave(reinterpret_cast<const void *>(kern[m]), resident[m]));
    for (int colour = 0; colour < 2; ++colour) {
        kern[m]<<<blocks, kThreads, 0, st>>>(k, colour, off);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lat

namespace lat {

bool resident_supported(const Geom &g)
{
    return wide_supported(g) && g.cpl == nullptr && resident_bytes(g) <= kResMaxBytes;
}

cudaError_t launch_sweep_resident(const Geom &g, int off, int n_sweeps, cudaStream_t st)
{
    const Geom k = tiled_geom(g);
    const size_t smem = resident_bytes(g);
    // Sites per thread: 4 (W = 1) while that keeps every thread busy, else 16.
    const bool narrow = (uint64_t)g.L * (g.half >> 2) <= (uint64_t)kResThreads;
    const int m = (g.model == LAT_NE ? 2 : 0) + (narrow ? 1 : 0);
    static bool attr[4] = {false, false, false, false};
    void (*fn[4])(Geom, int, int) = {k_resident<false, 4>, k_resident<false, 1>, k_resident<true, 4>,
                                     k_resident<true, 1>};
    if (!attr[m]) {
        cudaError_t e = cudaFuncSetAttribute(fn[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResMaxBytes);
        if (e != cudaSuccess) return e;
        attr[m] = true;
    }
    fn[m]<<<1, kResThreads, smem, st>>>(k, off, n_sweeps);
    return cudaGetLastError();
}

}  // namespace lat

namespace lat {

cudaError_t launch_batch_resident(const Geom *geoms, const long long *n, int n_lat, long long done, int chunk,
                                  size_t smem, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_batch_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kResMaxBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_batch_resident<<<n_lat, kResThreads, smem, st>>>(geoms, n, done, chunk);
    return cudaGetLastError();
}

size_t resident_smem_bytes(const Geom &g) { return resident_bytes(g); }

}  // namespace lat

namespace lat {

int wide_items(const Geom &g)
{
    const uint64_t chunks = (uint64_t)g.L * (g.half >> 4);
    const uint64_t per = (uint64_t)kItemChunks * kThreads;
    return (int)((chunks + per - 1) / per);
}

int batch_wide_grid(bool ne)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ne) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_wide<true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_wide<false>, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_wide(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item, int colour,
                              bool ne, int grid, cudaStream_t st)
{
    if (ne) k_batch_wide<true><<<grid, kThreads, 0, st>>>(geoms, items, n_items, next_item, colour);
    else k_batch_wide<false><<<grid, kThreads, 0, st>>>(geoms, items, n_items, next_item, colour);
    return cudaGetLastError();
}

}  // namespace lat
