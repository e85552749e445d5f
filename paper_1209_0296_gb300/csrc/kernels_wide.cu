// kernels_wide.cu -- two launches per sweep (one per colour, the kernel
// boundary being the device-wide barrier of §III.A steps 6-7) for 2D
// spin-1/2 lattices (Ising and North-East), int8 spins of +-1 in the
// checkerboard-planar layout, L a multiple of 32.
//
// A thread owns 16 consecutive same-colour sites of one plane row (one
// 16-byte load = four Philox groups), so the loads, index arithmetic and
// Philox set-up are shared by 16 sites.  The colour-c sites only read the
// other plane, so the colour-c pass never reads a byte another thread
// writes.  Neighbour counts, thresholds and acceptance are those of the
// tiled kernel (bytes 0x01 / 0xFF, bit-sliced adder, t' = thr - 1 table).
//
// The solo kernels (k_wide_pipe for Ising, uniform or with per-bond and
// per-site disorder; k_wide_pipe_ne for the North-East model; k_any_pipe*
// for any even L) walk one chunk column per thread down the rows with two
// chunks in flight, so the Philox draws of one chunk (wide multiplies) and
// the Metropolis step of the other (logic) share each instruction block.
// They read s[sweep & 1] and write s[(sweep+1) & 1] without copying a
// plane: colour 1 takes the new colour-0 sites from the new buffer.  The
// resident kernels (wide_chunk, in place) keep the whole lattice in one
// CTA's shared memory.
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
// row y of the resident kernel's shared-memory lattice, in place (both
// buffer pointers of g are that array).  W = 4 is 16 sites per thread;
// smaller W on small lattices gives more threads with shorter dependency
// chains.  kPre: the chunk's draws come from the caller (upre).
template <bool kNE, int W = 4, bool kPre = false>
LAT_D void wide_chunk(const SweepView g, const uint32_t *sthr, int colour, unsigned long long sweep,
                      const PhiloxPre &pp, int y, int k, Counts &cnt, const U4 *upre = nullptr)
{
    const int8_t *src = g.s0;
    int8_t *dst = g.s0;
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
    U4 u[W];
#pragma unroll
    for (int w = 0; w < W; ++w) u[w] = U4{0, 0, 0, 0};
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
    } else if (need) {
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

// ---------------------------------------------------------------------
// Software-pipelined two-launch Ising sweep, uniform or with per-bond
// coupling signs (kCpl) and per-site field signs (kFld).  Same chunks,
// draws, table and bits as the resident kernel's wide_chunk; the difference
// is the schedule.  A chunk costs two kinds of work that load
// different pipes: its four Philox4x32-10 calls (wide multiplies on the
// FMA pipe) and the Metropolis step (logic on the ALU pipe).  Done one
// after the other they keep one pipe idle while the other works, so each
// iteration here loads and draws chunk i+1 in the same straight-line block
// as the Metropolis step of chunk i, and the two streams interleave.
// ---------------------------------------------------------------------
struct WideIn {
    uint32_t S[4], O[4], U[4], D[4];
    uint32_t adj;
    uint32_t C[4];   // disorder bytes of the chunk's sites (kCpl only)
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
    const int8_t *pC;      // this colour's disorder bytes, + 16k (or null)
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
    c.pC = g.cpl ? reinterpret_cast<const int8_t *>(g.cpl) + (size_t)kColour * plane + 16 * k : nullptr;
    c.half = g.half;
    c.L = (uint32_t)g.L;
    c.G = g.G;
    c.k = k;
    const uint32_t nwr = g.half >> 2;   // 4-byte words per plane row
    c.adjb0 = 4u * wrap_once(4u * k - 1u + nwr, nwr);   // x = 2j: west word before the chunk
    c.adjb1 = 4u * wrap_once(4u * k + 4u, nwr);         // x = 2j+1: east word after it
    return c;
}

// Loads of the walk's chunk in plane row y (and its disorder bytes when kCpl).
template <int kColour, bool kCpl = false>
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
    if constexpr (kCpl) load_words<4>(c.pC + oy, in.C);
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
// sites (and the overlap with the reference when kRef); with kFld each
// colour adds the field sum of its own sites.
template <int kColour, bool kRef, bool kCpl = false, bool kFld = false>
LAT_D void col_step(const ColWalk<kColour> &c, const uint32_t *sthr, uint32_t y, const WideIn &in,
                    const U4 (&u)[4], Counts &cnt)
{
    const uint32_t oy = y * c.half;
    const bool p1 = ((kColour + y) & 1) != 0;
    const char *tb = reinterpret_cast<const char *>(sthr);
    const uint32_t M1 = 0x02020202u;
    uint32_t Sn[4], ue = 0, dn = 0, ed = 0;
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
        uint32_t Uw = in.U[w], Dw = in.D[w];
        if constexpr (kCpl) {
            // Eq. 1 couplings: a negative bond enters as a flipped neighbour
            // (XOR 0xFE turns +1 into -1 and back); bits 0-3 of a disorder
            // byte are the west, east, north and south bonds
            const uint32_t Cw = in.C[w];
            Lf ^= (Cw & 0x01010101u) * 0xFEu;
            R ^= ((Cw >> 1) & 0x01010101u) * 0xFEu;
            Uw ^= ((Cw >> 2) & 0x01010101u) * 0xFEu;
            Dw ^= ((Cw >> 3) & 0x01010101u) * 0xFEu;
        }
        const uint32_t s1 = Uw ^ Dw ^ Lf;
        const uint32_t c1 = (Uw & Dw) | (Uw & Lf) | (Dw & Lf);
        const uint32_t b0 = s1 ^ R;
        const uint32_t b1 = c1 ^ (s1 & R);
        const uint32_t b2 = c1 & s1 & R;
        uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) | (in.S[w] & 0x20202020u);
        if constexpr (kFld) idx |= in.C[w] & 0x40404040u;   // eta_i = -1: the -h entries 16..31
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
        // eta_i s_i is down when exactly one of (s_i down: bit 1, eta_i = -1: bit 6) holds
        if constexpr (kFld) ed += (Sn[w] ^ (in.C[w] >> 5)) & M1;
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
    if constexpr (kFld) cnt.fld += 16 - byte_sum(ed);
}

constexpr int kPipeMinB = 2;   // CTAs per SM (the two chunks in flight need ~100 registers)

// kFld: a 32-entry table, entries 16..31 built from the -h half of the full
// table (t' = thr - 1 form, all ones = always), index sd << 3 | nd as for
// entries 0..15.
template <int kColour, bool kRef, bool kCpl = false, bool kFld = false>
__global__ void __launch_bounds__(kThreads, kPipeMinB) k_wide_pipe(Geom g, int off)
{
    __shared__ uint32_t sthr[kFld ? 32 : 16];
    __shared__ int red[kThreads / 32][5];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    if constexpr (kFld) {
        if (threadIdx.x >= 16 && threadIdx.x < 32) {
            const int e = threadIdx.x - 16, nd = e & 7;
            uint32_t t = 0u;
            if (nd <= 4) {
                const int ds = (e >> 3) ? 2 : -2, n = 4 - 2 * nd;
                const TabEntry te = g.tab[(2 * g.dsmax + 1) * g.nn + (ds + g.dsmax) * g.nn + (n + g.nmax)];
                t = te.always ? 0xFFFFFFFFu : te.thr - 1u;
            }
            sthr[threadIdx.x] = t;
        }
    }
    __syncthreads();
    dep_wait();
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
        col_load<kColour, kCpl>(c, y, A);
        col_draws<kColour>(pp, c, y, uA);
        for (;;) {
            const uint32_t y1 = y + rs;
            if (y1 >= L) {
                col_step<kColour, kRef, kCpl, kFld>(c, sthr, y, A, uA, cnt);
                break;
            }
            col_load<kColour, kCpl>(c, y1, B);
            col_draws<kColour>(pp, c, y1, uB);
            col_step<kColour, kRef, kCpl, kFld>(c, sthr, y, A, uA, cnt);
            const uint32_t y2 = y1 + rs;
            if (y2 >= L) {
                col_step<kColour, kRef, kCpl, kFld>(c, sthr, y1, B, uB, cnt);
                break;
            }
            col_load<kColour, kCpl>(c, y2, A);
            col_draws<kColour>(pp, c, y2, uA);
            col_step<kColour, kRef, kCpl, kFld>(c, sthr, y1, B, uB, cnt);
            y = y2;
        }
    }
    dep_launch();   // main work done: the next kernel may be scheduled
    if constexpr (kColour == 1) flush(v, sweep, cnt, false, red);
    if constexpr (kFld) flush_one(fld_slot(g.ctrl, sweep), cnt.fld, red);   // both colours
}

// ---------------------------------------------------------------------
// North-East model (§III.B), the same column walk with the loads of the
// next chunk in flight, and draws compacted across the warp.  A site moves
// only if its north and east neighbours are up, and then, in c-mode with
// c < 1/2, an up site turns down without a draw; so only a few percent of
// the Philox groups need a draw.  Each lane marks the groups of its chunk
// that do; the warp lists them (ballot and prefix count), every lane makes
// the Philox calls of list entries lane, lane + 32, ... and the draws go
// back to their owners through shared memory.  A warp then makes
// ceil(needed / 32) calls per lane instead of 4.  Same groups, counters and
// bits as the other kernels.
// ---------------------------------------------------------------------
constexpr int kNeSlots = 4 * 32;   // list entries per warp (4 groups per lane)

// kCMode: the c-mode rates of §III.B depend on the move alone, not on the
// neighbour sum (every neighbour-count entry of a row of the table is the
// same), so the index skips the neighbour-count bits (colour 0 then needs no
// neighbour adder at all; colour 1 keeps it for the bond count).
template <int kColour, bool kRef, bool kCMode = false>
LAT_D void ne_col_step(bool act, const ColWalk<kColour> &c, const uint8_t *fl_c, const uint8_t *fl_o,
                       const uint32_t *sthr, uint32_t y, const WideIn &in, const PhiloxPre &pp,
                       uint32_t *gtab, uint4 *dq, Counts &cnt)
{
    const uint32_t oy = y * c.half;
    const bool p1 = ((kColour + y) & 1) != 0;
    const char *tb = reinterpret_cast<const char *>(sthr);
    const uint32_t M1 = 0x02020202u;
    const int lane = threadIdx.x & 31;
    uint32_t Lf[4], R[4], t[4][4], locked[4], s1[4], c1[4];
    unsigned need = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (!p1) {
            Lf[w] = __funnelshift_l(w == 0 ? in.adj : in.O[w - 1], in.O[w], 8);
            R[w] = in.O[w];
        } else {
            Lf[w] = in.O[w];
            R[w] = __funnelshift_r(in.O[w], w == 3 ? in.adj : in.O[w + 1], 8);
        }
        const uint32_t Uw = in.U[w], Dw = in.D[w];
        s1[w] = Uw ^ Dw ^ Lf[w];
        c1[w] = (Uw & Dw) | (Uw & Lf[w]) | (Dw & Lf[w]);
        const uint32_t b0 = s1[w] ^ R[w];
        const uint32_t b1 = c1[w] ^ (s1[w] & R[w]);
        const uint32_t b2 = c1[w] & s1[w] & R[w];
        // §III.B: north (U) and east (R) must be up.  A locked site (either
        // down: bit 6 of U | R set) indexes entries 16..31 of the table, all
        // t' = all ones, so it needs no draw; its flip is masked off below.
        locked[w] = Uw | R[w];
        const uint32_t idx = kCMode ? (in.S[w] & 0x20202020u) | (locked[w] & 0x40404040u)
                                    : (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) |
                                          (in.S[w] & 0x20202020u) | (locked[w] & 0x40404040u);
        t[w][0] = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
        t[w][1] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
        t[w][2] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
        t[w][3] = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
        if (act && (t[w][0] & t[w][1] & t[w][2] & t[w][3]) != 0xFFFFFFFFu) need |= 1u << w;
    }
    // the warp's list of groups that need a draw: group w of every lane, then w+1
    unsigned bal[4], base[4], total = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        bal[w] = __ballot_sync(0xffffffffu, (need >> w) & 1u);
        base[w] = total;
        total += __popc(bal[w]);
    }
    U4 u[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) u[w] = U4{0u, 0u, 0u, 0u};   // t' all ones: any draw accepts
    if (total > 0) {   // warp-uniform
        const unsigned lt_mask = (1u << lane) - 1u;
        const uint32_t g0 = y * c.G + 4u * c.k;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if ((need >> w) & 1u) gtab[base[w] + __popc(bal[w] & lt_mask)] = g0 + (uint32_t)w;
        __syncwarp();
        for (unsigned j = (unsigned)lane; j < total; j += 32) {
            const U4 d = philox_item(pp, gtab[j], (uint32_t)kColour);
            dq[j] = make_uint4(d.x, d.y, d.z, d.w);
        }
        __syncwarp();
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if ((need >> w) & 1u) {
                const uint4 q = dq[base[w] + __popc(bal[w] & lt_mask)];
                u[w] = U4{q.x, q.y, q.z, q.w};
            }
        __syncwarp();   // the next chunk's list may overwrite these entries
    }
    if (!act) return;
    uint32_t Sn[4], ue = 0, dn = 0, chg = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t acc = (u[w].x <= t[w][0] ? 1u : 0u) | (u[w].y <= t[w][1] ? 2u : 0u) |
                             (u[w].z <= t[w][2] ? 4u : 0u) | (u[w].w <= t[w][3] ? 8u : 0u);
        const uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu & ~locked[w];
        chg |= ((((F >> 1) & 0x01010101u) * 0x01020408u) >> 24 & 0xFu) << (8 * w);
        Sn[w] = in.S[w] ^ F;
        if constexpr (kColour == 1) {
            ue += ((s1[w] ^ Sn[w]) & M1) + ((c1[w] ^ Sn[w]) & 0x04040404u) + ((R[w] ^ Sn[w]) & M1);
            dn += (Sn[w] & M1) + (in.O[w] & M1);
        }
    }
    store_words<4>(c.dS + oy, Sn);
    // persistence bytes of the chunk's four groups (bit q = site 4m+q)
    uint32_t *fp = reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(fl_c) + (size_t)y * c.G);
    const uint32_t f = *fp | chg;
    *fp = f;
    if constexpr (kColour == 1) {
        const uint32_t fo = *reinterpret_cast<const uint32_t *>(fl_o + (size_t)y * c.G);
        const int d2 = byte_sum(dn);
        cnt.bond += 64 - byte_sum(ue);
        cnt.mag += 32 - d2;
        cnt.up += 32 - (d2 >> 1);
        cnt.unfl += 32 - __popc(f) - __popc(fo);
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

template <int kColour, bool kRef, bool kCMode = false>
__global__ void __launch_bounds__(kThreads, kPipeMinB) k_wide_pipe_ne(Geom g, int off)
{
    __shared__ uint32_t sthr[32];   // entries 16..31: locked sites, always accepted (then masked)
    __shared__ int red[kThreads / 32][5];
    __shared__ uint32_t gtab[kThreads / 32][kNeSlots];
    __shared__ uint4 dq[kThreads / 32][kNeSlots];
    if (threadIdx.x < 32) sthr[threadIdx.x] = threadIdx.x < 16 ? g.thr16[threadIdx.x] : 0xFFFFFFFFu;
    __syncthreads();
    dep_wait();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const SweepView v = sweep_view(g);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    Counts cnt;
    const uint32_t cpr = g.half >> 4;
    const uint32_t rs = (gridDim.x * blockDim.x) / cpr;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t L = (uint32_t)g.L;
    uint32_t y = gt / cpr;
    const uint32_t k = gt - y * cpr;
    bool act = y < rs && y < L;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const ColWalk<kColour> c = col_walk<kColour>(v, old, nw, act ? k : 0u);
    const uint8_t *fl_c = g.flags + (size_t)kColour * g.rows * g.G + 4u * k;
    const uint8_t *fl_o = g.flags + (size_t)(1 - kColour) * g.rows * g.G + 4u * k;
    const int warp = threadIdx.x >> 5;
    // Two chunks in flight (A and B in turn).  The warp's lanes stay in step
    // (the draw list is made by the whole warp), so a lane that has run out
    // of rows takes part with nothing to update.
    WideIn A, B;
    if (act) col_load<kColour>(c, y, A);
    for (;;) {
        if (!__any_sync(0xffffffffu, act)) break;
        const uint32_t y1 = y + rs;
        const bool act1 = act && y1 < L;
        if (act1) col_load<kColour>(c, y1, B);
        ne_col_step<kColour, kRef, kCMode>(act, c, fl_c, fl_o, sthr, y, A, pp, gtab[warp], dq[warp], cnt);
        if (!__any_sync(0xffffffffu, act1)) break;
        const uint32_t y2 = y1 + rs;
        const bool act2 = act1 && y2 < L;
        if (act2) col_load<kColour>(c, y2, A);
        ne_col_step<kColour, kRef, kCMode>(act1, c, fl_c, fl_o, sthr, y1, B, pp, gtab[warp], dq[warp], cnt);
        y = y2;
        act = act2;
    }
    dep_launch();   // main work done: the next kernel may be scheduled
    if constexpr (kColour == 1) flush(v, sweep, cnt, true, red);
}

// ---------------------------------------------------------------------
// Any even L, 16 sites per lane: the wide kernel's chunk of four Philox
// groups on rows at any byte alignment.  A chunk's 16 bytes are gathered
// from the aligned words that hold them; the last chunk of a row holds
// L/2 % 16 sites (its bytes past the row are masked, its neighbour past the
// row end is the row's first byte); stores write whole aligned words inside
// the chunk and single bytes at its two ends, so no byte of another lane's
// chunk is touched.  Column walk with two chunks in flight as in
// k_wide_pipe (Ising: the next chunk's draws too) and, for the North-East
// model, the warp-compacted draws of k_wide_pipe_ne.
// ---------------------------------------------------------------------

// Bytes p[0 .. nv) (1 <= nv <= 16) as four words, byte b = p[b], the bytes
// from nv on unspecified; an aligned word that holds none of them is not
// read (the spin buffers are multiples of 4 bytes, so every word read is in
// bounds).  kAligned: p is 16-byte aligned and nv = 16 (every chunk of a
// lattice with L % 32 == 0), one 16-byte load.
template <bool kAligned = false>
LAT_D void load16_any(const int8_t *p, uint32_t nv, uint32_t (&v)[4])
{
    if constexpr (kAligned) {
        load_words<4>(p, v);
        return;
    }
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t sh = (uint32_t)(a & 3u);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a - sh);
    uint32_t x[5];
    x[0] = w[0];
#pragma unroll
    for (int i = 1; i < 5; ++i) x[i] = (4u * (uint32_t)i < nv + sh) ? w[i] : 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __funnelshift_r(x[i], x[i + 1], 8u * sh);
}

// Write bytes [0, nv) of v to p (any alignment) and no other byte: whole
// aligned words where the chunk covers them, single bytes at its ends.
template <bool kAligned = false>
LAT_D void store16_any(int8_t *p, uint32_t nv, const uint32_t (&v)[4])
{
    if constexpr (kAligned) {
        store_words<4>(p, v);
        return;
    }
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t sh = (uint32_t)(a & 3u);
    uint32_t *w = reinterpret_cast<uint32_t *>(a - sh);
    uint32_t o[5];   // o[i]: the chunk's bytes that fall in aligned word i
    o[0] = __funnelshift_l(0u, v[0], 8u * sh);
#pragma unroll
    for (int i = 1; i < 4; ++i) o[i] = __funnelshift_l(v[i - 1], v[i], 8u * sh);
    o[4] = __funnelshift_l(v[3], 0u, 8u * sh);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int lo = i == 0 ? (int)sh : 0;
        const int hi = min(4, (int)(nv + sh) - 4 * i);
        if (hi <= lo) continue;
        if (lo == 0 && hi == 4) {
            w[i] = o[i];
        } else {
            int8_t *pb = reinterpret_cast<int8_t *>(w + i);
            for (int j = lo; j < hi; ++j) pb[j] = (int8_t)(o[i] >> (8 * j));
        }
    }
}

struct AnyIn {
    uint32_t S[4], O[4], U[4], D[4];
    uint32_t nb;   // the other plane's byte past the chunk's edge (west of j0, or east of its last site)
};

// One thread's column of chunks (chunk k of every plane row it visits).
template <int kColour>
struct AnyWalk {
    const int8_t *pS, *pO;   // planes: this colour's old sites, the other colour's current sites
    int8_t *dS;              // this colour's plane in the new buffer
    const int8_t *r1, *r0;   // reference planes 1 and 0 (or null)
    uint32_t half, L, G, k, j0, nv;
    uint32_t vm[4];          // valid-byte masks of the chunk's words
    uint32_t jprev, jnext;   // row index of the west neighbour of j0 / the east neighbour of the last site
};

template <int kColour>
LAT_D AnyWalk<kColour> any_walk(const SweepView &g, const int8_t *old, int8_t *nw, uint32_t k)
{
    constexpr int oc = 1 - kColour;
    AnyWalk<kColour> c;
    const uint32_t plane = (uint32_t)g.plane;
    c.pS = old + (size_t)kColour * plane;
    c.pO = (kColour == 0 ? old : nw) + (size_t)oc * plane;
    c.dS = nw + (size_t)kColour * plane;
    c.r1 = g.ref ? g.ref + (size_t)plane : nullptr;
    c.r0 = g.ref;
    c.half = g.half;
    c.L = (uint32_t)g.L;
    c.G = g.G;
    c.k = k;
    c.j0 = 16u * k;
    c.nv = min(16u, g.half - c.j0);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int n = (int)c.nv - 4 * w;
        c.vm[w] = n >= 4 ? 0xFFFFFFFFu : (n <= 0 ? 0u : (1u << (8 * n)) - 1u);
    }
    c.jprev = c.j0 == 0u ? g.half - 1u : c.j0 - 1u;
    c.jnext = c.j0 + c.nv == g.half ? 0u : c.j0 + c.nv;
    return c;
}

template <int kColour, bool kAligned = false>
LAT_D void any_load(const AnyWalk<kColour> &c, uint32_t y, AnyIn &in)
{
    const uint32_t oy = y * c.half;
    const uint32_t oym = y == 0 ? oy + (c.L - 1) * c.half : oy - c.half;
    const uint32_t oyp = y == c.L - 1 ? 0u : oy + c.half;
    load16_any<kAligned>(c.pS + oy + c.j0, c.nv, in.S);
    load16_any<kAligned>(c.pO + oy + c.j0, c.nv, in.O);
    load16_any<kAligned>(c.pO + oym + c.j0, c.nv, in.U);   // north
    load16_any<kAligned>(c.pO + oyp + c.j0, c.nv, in.D);   // south
    in.nb = (uint32_t)(uint8_t)c.pO[oy + (((kColour + y) & 1) ? c.jnext : c.jprev)];
}

template <int kColour>
LAT_D void any_draws(const PhiloxPre &pp, const AnyWalk<kColour> &c, uint32_t y, U4 (&u)[4])
{
    const uint32_t g0 = y * c.G + 4u * c.k;
#pragma unroll
    for (int w = 0; w < 4; ++w) u[w] = philox_item(pp, g0 + (uint32_t)w, (uint32_t)kColour);
}

// West (Lf) and east (R) neighbour words of the chunk's sites.
template <int kColour>
LAT_D void any_sides(const AnyWalk<kColour> &c, uint32_t y, const AnyIn &in, uint32_t (&Lf)[4], uint32_t (&R)[4])
{
    if (((kColour + y) & 1) == 0) {   // x = 2j: west is j-1 (nb for j0), east is j
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            Lf[w] = __funnelshift_l(w == 0 ? (in.nb << 24) : in.O[w - 1], in.O[w], 8);
            R[w] = in.O[w];
        }
    } else {                          // x = 2j+1: west is j, east is j+1 (nb for the last site)
        // a partial chunk's last site: its east neighbour nb goes to byte nv
        // of the sequence (a mask that is zero in every other word)
        uint32_t Oe[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t d = c.nv - 4u * (uint32_t)w;
            const uint32_t m = d < 4u ? (0xFFu << (8u * d)) : 0u;
            Oe[w] = (in.O[w] & ~m) | ((in.nb << (8u * (d & 3u))) & m);
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            Lf[w] = in.O[w];
            R[w] = __funnelshift_r(Oe[w], w == 3 ? in.nb : Oe[w + 1], 8);
        }
    }
}

template <int kColour, bool kRef, bool kAligned = false>
LAT_D void any_step(const AnyWalk<kColour> &c, const uint32_t *sthr, uint32_t y, const AnyIn &in, const U4 (&u)[4],
                    Counts &cnt)
{
    const uint32_t oy = y * c.half;
    const char *tb = reinterpret_cast<const char *>(sthr);
    const uint32_t M1 = 0x02020202u;
    uint32_t Lf[4], R[4];
    any_sides<kColour>(c, y, in, Lf, R);
    uint32_t Sn[4], ue = 0, dn = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t Uw = in.U[w], Dw = in.D[w];
        const uint32_t s1 = Uw ^ Dw ^ Lf[w];
        const uint32_t c1 = (Uw & Dw) | (Uw & Lf[w]) | (Dw & Lf[w]);
        const uint32_t b0 = s1 ^ R[w];
        const uint32_t b1 = c1 ^ (s1 & R[w]);
        const uint32_t b2 = c1 & s1 & R[w];
        const uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) | (in.S[w] & 0x20202020u);
        const uint32_t t0 = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
        const uint32_t t1 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
        const uint32_t t2 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
        const uint32_t t3 = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
        const uint32_t acc = (u[w].x <= t0 ? 1u : 0u) | (u[w].y <= t1 ? 2u : 0u) | (u[w].z <= t2 ? 4u : 0u) |
                             (u[w].w <= t3 ? 8u : 0u);
        const uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu & c.vm[w];
        Sn[w] = in.S[w] ^ F;
        if constexpr (kColour == 1) {
            ue += (((s1 ^ Sn[w]) & M1) + ((c1 ^ Sn[w]) & 0x04040404u) + ((R[w] ^ Sn[w]) & M1)) & c.vm[w];
            dn += ((Sn[w] & M1) + (in.O[w] & M1)) & c.vm[w];
        }
    }
    store16_any<kAligned>(c.dS + oy + c.j0, c.nv, Sn);
    if constexpr (kColour == 1) {
        const int nv = (int)c.nv;
        const int d2 = byte_sum(dn);
        cnt.bond += 4 * nv - byte_sum(ue);
        cnt.mag += 2 * nv - d2;
        cnt.up += 2 * nv - (d2 >> 1);
        if constexpr (kRef) {
            uint32_t R1[4], R0[4], dr = 0;
            load16_any<kAligned>(c.r1 + oy + c.j0, c.nv, R1);
            load16_any<kAligned>(c.r0 + oy + c.j0, c.nv, R0);
#pragma unroll
            for (int w = 0; w < 4; ++w) dr += (((Sn[w] ^ R1[w]) & M1) + ((in.O[w] ^ R0[w]) & M1)) & c.vm[w];
            cnt.acf += 2 * nv - byte_sum(dr);
        }
    }
}

template <int kColour, bool kRef>
__global__ void __launch_bounds__(kThreads, kPipeMinB) k_any_pipe(Geom g, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][5];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    dep_wait();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const SweepView v = sweep_view(g);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    Counts cnt;
    const uint32_t cpr = (g.half + 15u) >> 4;   // chunks per plane row, the last partial
    const uint32_t rs = (gridDim.x * blockDim.x) / cpr;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t y = gt / cpr;
    const uint32_t k = gt - y * cpr;
    if (y < rs && y < (uint32_t)g.L) {
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        const AnyWalk<kColour> c = any_walk<kColour>(v, old, nw, k);
        const uint32_t L = (uint32_t)g.L;
        AnyIn A, B;
        U4 uA[4], uB[4];
        any_load<kColour>(c, y, A);
        any_draws<kColour>(pp, c, y, uA);
        for (;;) {
            const uint32_t y1 = y + rs;
            if (y1 >= L) {
                any_step<kColour, kRef>(c, sthr, y, A, uA, cnt);
                break;
            }
            any_load<kColour>(c, y1, B);
            any_draws<kColour>(pp, c, y1, uB);
            any_step<kColour, kRef>(c, sthr, y, A, uA, cnt);
            const uint32_t y2 = y1 + rs;
            if (y2 >= L) {
                any_step<kColour, kRef>(c, sthr, y1, B, uB, cnt);
                break;
            }
            any_load<kColour>(c, y2, A);
            any_draws<kColour>(pp, c, y2, uA);
            any_step<kColour, kRef>(c, sthr, y1, B, uB, cnt);
            y = y2;
        }
    }
    dep_launch();   // main work done: the next kernel may be scheduled
    if constexpr (kColour == 1) flush(v, sweep, cnt, false, red);
}

// North-East at any even L: the step of ne_col_step with any-alignment
// loads and stores, per-byte persistence updates (the groups of a row need
// not start on a word), and the warp-compacted draws.
template <int kColour, bool kRef, bool kAligned = false, bool kCMode = false>
LAT_D void any_ne_step(bool act, const AnyWalk<kColour> &c, uint8_t *fl_c, const uint8_t *fl_o,
                       const uint32_t *sthr, uint32_t y, const AnyIn &in, const PhiloxPre &pp, uint32_t *gtab,
                       uint4 *dq, Counts &cnt)
{
    const uint32_t oy = y * c.half;
    const char *tb = reinterpret_cast<const char *>(sthr);
    const uint32_t M1 = 0x02020202u;
    const int lane = threadIdx.x & 31;
    uint32_t Lf[4], R[4], t[4][4], locked[4], s1[4], c1[4];
    any_sides<kColour>(c, y, in, Lf, R);
    unsigned need = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t Uw = in.U[w], Dw = in.D[w];
        s1[w] = Uw ^ Dw ^ Lf[w];
        c1[w] = (Uw & Dw) | (Uw & Lf[w]) | (Dw & Lf[w]);
        const uint32_t b0 = s1[w] ^ R[w];
        const uint32_t b1 = c1[w] ^ (s1[w] & R[w]);
        const uint32_t b2 = c1[w] & s1[w] & R[w];
        // §III.B: a locked site (north or east down) indexes the all-accept
        // entries 16..31; so do the bytes past the row (masked below)
        locked[w] = Uw | R[w] | ~c.vm[w];
        const uint32_t idx = kCMode ? (in.S[w] & 0x20202020u) | (locked[w] & 0x40404040u)
                                    : (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) |
                                          (in.S[w] & 0x20202020u) | (locked[w] & 0x40404040u);
        t[w][0] = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
        t[w][1] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
        t[w][2] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
        t[w][3] = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
        if (act && (t[w][0] & t[w][1] & t[w][2] & t[w][3]) != 0xFFFFFFFFu) need |= 1u << w;
    }
    unsigned bal[4], base[4], total = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        bal[w] = __ballot_sync(0xffffffffu, (need >> w) & 1u);
        base[w] = total;
        total += __popc(bal[w]);
    }
    U4 u[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) u[w] = U4{0u, 0u, 0u, 0u};
    if (total > 0) {
        const unsigned lt_mask = (1u << lane) - 1u;
        const uint32_t g0 = y * c.G + 4u * c.k;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if ((need >> w) & 1u) gtab[base[w] + __popc(bal[w] & lt_mask)] = g0 + (uint32_t)w;
        __syncwarp();
        for (unsigned j = (unsigned)lane; j < total; j += 32) {
            const U4 d = philox_item(pp, gtab[j], (uint32_t)kColour);
            dq[j] = make_uint4(d.x, d.y, d.z, d.w);
        }
        __syncwarp();
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if ((need >> w) & 1u) {
                const uint4 q = dq[base[w] + __popc(bal[w] & lt_mask)];
                u[w] = U4{q.x, q.y, q.z, q.w};
            }
        __syncwarp();
    }
    if (!act) return;
    uint32_t Sn[4], ue = 0, dn = 0, chg = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t acc = (u[w].x <= t[w][0] ? 1u : 0u) | (u[w].y <= t[w][1] ? 2u : 0u) |
                             (u[w].z <= t[w][2] ? 4u : 0u) | (u[w].w <= t[w][3] ? 8u : 0u);
        const uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu & ~locked[w];
        chg |= ((((F >> 1) & 0x01010101u) * 0x01020408u) >> 24 & 0xFu) << (8 * w);
        Sn[w] = in.S[w] ^ F;
        if constexpr (kColour == 1) {
            ue += (((s1[w] ^ Sn[w]) & M1) + ((c1[w] ^ Sn[w]) & 0x04040404u) + ((R[w] ^ Sn[w]) & M1)) & c.vm[w];
            dn += ((Sn[w] & M1) + (in.O[w] & M1)) & c.vm[w];
        }
    }
    store16_any<kAligned>(c.dS + oy + c.j0, c.nv, Sn);
    // persistence bytes of the chunk's groups that exist (4k + w < G)
    uint8_t *fp = fl_c + (size_t)y * c.G;
    const uint8_t *fop = fl_o + (size_t)y * c.G;
    const uint32_t ng = min(4u, c.G - 4u * c.k);
    int fpop = 0, fopop = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if ((uint32_t)w < ng) {
            const uint32_t f = (uint32_t)fp[w] | ((chg >> (8 * w)) & 0xFu);
            fp[w] = (uint8_t)f;
            fpop += __popc(f);
            if constexpr (kColour == 1) fopop += __popc((uint32_t)fop[w]);
        }
    if constexpr (kColour == 1) {
        const int nv = (int)c.nv;
        const int d2 = byte_sum(dn);
        cnt.bond += 4 * nv - byte_sum(ue);
        cnt.mag += 2 * nv - d2;
        cnt.up += 2 * nv - (d2 >> 1);
        cnt.unfl += 2 * nv - fpop - fopop;
        if constexpr (kRef) {
            uint32_t R1[4], R0[4], dr = 0;
            load16_any<kAligned>(c.r1 + oy + c.j0, c.nv, R1);
            load16_any<kAligned>(c.r0 + oy + c.j0, c.nv, R0);
#pragma unroll
            for (int w = 0; w < 4; ++w) dr += (((Sn[w] ^ R1[w]) & M1) + ((in.O[w] ^ R0[w]) & M1)) & c.vm[w];
            cnt.acf += 2 * nv - byte_sum(dr);
        }
    }
}

template <int kColour, bool kRef, bool kCMode = false>
__global__ void __launch_bounds__(kThreads, kPipeMinB) k_any_pipe_ne(Geom g, int off)
{
    __shared__ uint32_t sthr[32];   // entries 16..31: locked sites, always accepted (then masked)
    __shared__ int red[kThreads / 32][5];
    __shared__ uint32_t gtab[kThreads / 32][kNeSlots];
    __shared__ uint4 dq[kThreads / 32][kNeSlots];
    if (threadIdx.x < 32) sthr[threadIdx.x] = threadIdx.x < 16 ? g.thr16[threadIdx.x] : 0xFFFFFFFFu;
    __syncthreads();
    dep_wait();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const SweepView v = sweep_view(g);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    Counts cnt;
    const uint32_t cpr = (g.half + 15u) >> 4;
    const uint32_t rs = (gridDim.x * blockDim.x) / cpr;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t L = (uint32_t)g.L;
    uint32_t y = gt / cpr;
    const uint32_t k = gt - y * cpr;
    bool act = y < rs && y < L;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const AnyWalk<kColour> c = any_walk<kColour>(v, old, nw, act ? k : 0u);
    uint8_t *fl_c = g.flags + (size_t)kColour * g.rows * g.G + 4u * c.k;
    const uint8_t *fl_o = g.flags + (size_t)(1 - kColour) * g.rows * g.G + 4u * c.k;
    const int warp = threadIdx.x >> 5;
    AnyIn A, B;
    if (act) any_load<kColour>(c, y, A);
    for (;;) {
        if (!__any_sync(0xffffffffu, act)) break;
        const uint32_t y1 = y + rs;
        const bool act1 = act && y1 < L;
        if (act1) any_load<kColour>(c, y1, B);
        any_ne_step<kColour, kRef, false, kCMode>(act, c, fl_c, fl_o, sthr, y, A, pp, gtab[warp], dq[warp], cnt);
        if (!__any_sync(0xffffffffu, act1)) break;
        const uint32_t y2 = y1 + rs;
        const bool act2 = act1 && y2 < L;
        if (act2) any_load<kColour>(c, y2, A);
        any_ne_step<kColour, kRef, false, kCMode>(act1, c, fl_c, fl_o, sthr, y1, B, pp, gtab[warp], dq[warp], cnt);
        y = y2;
        act = act2;
    }
    dep_launch();   // main work done: the next kernel may be scheduled
    if constexpr (kColour == 1) flush(v, sweep, cnt, true, red);
}

// Batched form of the any-L kernels: a persistent grid takes (lattice,
// item) pairs from an atomic counter.  An item is a band of rows and, in
// rows of more than 256 chunks, a segment of 256 chunk columns; a thread
// walks one chunk column down the band with two chunks in flight, as the
// solo kernels do.
struct AnyItemShape {
    uint32_t cpr, nseg, rsb, br;   // chunks per row, column segments, rows per pass, rows per band
};

// Rows a thread visits per item (passes): given by the batch (its tuner),
// or 0 for the default: 8 on large lattices (few items, long pipelines), 2
// on small ones (enough items to spread a batch of small lattices over the
// SMs).
LAT_HD AnyItemShape any_item_shape(uint32_t half, uint32_t passes)
{
    AnyItemShape sh;
    sh.cpr = (half + 15u) >> 4;
    sh.nseg = (sh.cpr + kThreads - 1u) / kThreads;
    sh.rsb = sh.cpr <= (uint32_t)kThreads ? (uint32_t)kThreads / sh.cpr : 1u;
    if (passes == 0u) passes = half >= 512u ? 8u : 2u;
    sh.br = passes * sh.rsb;
    return sh;
}

template <int kColour, bool kNE, bool kAligned, bool kCMode>
LAT_D void batch_any_item(const SweepView &v, const uint32_t *sthr, uint32_t item, uint32_t passes, uint32_t *gtab,
                          uint4 *dq, Counts &cnt)
{
    const unsigned long long sweep = v.ctrl->sweep;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), v.key0, v.key1);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    const AnyItemShape sh = any_item_shape(v.half, passes);
    const uint32_t L = (uint32_t)v.L;
    const uint32_t band = item / sh.nseg, seg = item - band * sh.nseg;
    const uint32_t y0 = band * sh.br, y1 = min(L, y0 + sh.br);
    uint32_t k, r0;
    if (sh.cpr <= (uint32_t)kThreads) {
        k = threadIdx.x % sh.cpr;
        r0 = threadIdx.x / sh.cpr;
    } else {
        k = seg * kThreads + threadIdx.x;
        r0 = 0;
    }
    const bool mine = k < sh.cpr && r0 < sh.rsb;
    uint32_t y = y0 + r0;
    const AnyWalk<kColour> c = any_walk<kColour>(v, old, nw, mine ? k : 0u);
    if constexpr (!kNE) {
        if (!(mine && y < y1)) return;
        AnyIn A, B;
        U4 uA[4], uB[4];
        any_load<kColour, kAligned>(c, y, A);
        any_draws<kColour>(pp, c, y, uA);
        for (;;) {
            const uint32_t ya = y + sh.rsb;
            if (ya >= y1) {
                if (v.ref) any_step<kColour, true, kAligned>(c, sthr, y, A, uA, cnt);
                else any_step<kColour, false, kAligned>(c, sthr, y, A, uA, cnt);
                break;
            }
            any_load<kColour, kAligned>(c, ya, B);
            any_draws<kColour>(pp, c, ya, uB);
            if (v.ref) any_step<kColour, true, kAligned>(c, sthr, y, A, uA, cnt);
            else any_step<kColour, false, kAligned>(c, sthr, y, A, uA, cnt);
            const uint32_t yb = ya + sh.rsb;
            if (yb >= y1) {
                if (v.ref) any_step<kColour, true, kAligned>(c, sthr, ya, B, uB, cnt);
                else any_step<kColour, false, kAligned>(c, sthr, ya, B, uB, cnt);
                break;
            }
            any_load<kColour, kAligned>(c, yb, A);
            any_draws<kColour>(pp, c, yb, uA);
            if (v.ref) any_step<kColour, true, kAligned>(c, sthr, ya, B, uB, cnt);
            else any_step<kColour, false, kAligned>(c, sthr, ya, B, uB, cnt);
            y = yb;
        }
    } else {
        // the warp's lanes stay in step (warp-compacted draws)
        uint8_t *fl_c = v.flags + (size_t)kColour * v.rows * v.G + 4u * c.k;
        const uint8_t *fl_o = v.flags + (size_t)(1 - kColour) * v.rows * v.G + 4u * c.k;
        bool act = mine && y < y1;
        AnyIn A, B;   // two chunks in flight
        if (act) any_load<kColour, kAligned>(c, y, A);
        for (;;) {
            if (!__any_sync(0xffffffffu, act)) break;
            const uint32_t ya = y + sh.rsb;
            const bool act1 = act && ya < y1;
            if (act1) any_load<kColour, kAligned>(c, ya, B);
            if (v.ref) any_ne_step<kColour, true, kAligned, kCMode>(act, c, fl_c, fl_o, sthr, y, A, pp, gtab, dq, cnt);
            else any_ne_step<kColour, false, kAligned, kCMode>(act, c, fl_c, fl_o, sthr, y, A, pp, gtab, dq, cnt);
            if (!__any_sync(0xffffffffu, act1)) break;
            const uint32_t yb = ya + sh.rsb;
            const bool act2 = act1 && yb < y1;
            if (act2) any_load<kColour, kAligned>(c, yb, A);
            if (v.ref) any_ne_step<kColour, true, kAligned, kCMode>(act1, c, fl_c, fl_o, sthr, ya, B, pp, gtab, dq, cnt);
            else any_ne_step<kColour, false, kAligned, kCMode>(act1, c, fl_c, fl_o, sthr, ya, B, pp, gtab, dq, cnt);
            y = yb;
            act = act2;
        }
    }
}

// kCMode: a list of c-mode North-East lattices (their steps skip the
// neighbour-count bits of the table index).
template <bool kNE, bool kAligned, int kColour, bool kCMode = false>
__global__ void __launch_bounds__(kThreads, kPipeMinB) k_batch_any(const Geom *geoms, const uint2 *items, int n_items,
                                                                  unsigned *next_item, uint32_t passes)
{
    __shared__ uint32_t sthr[32];   // entries 16..31: locked North-East sites
    __shared__ int red[kThreads / 32][5];
    __shared__ uint32_t gtab[kNE ? kThreads / 32 : 1][kNeSlots];
    __shared__ uint4 dq[kNE ? kThreads / 32 : 1][kNeSlots];
    __shared__ Geom sg;
    __shared__ int cur;
    int loaded = -1;
    const int warp = kNE ? (int)(threadIdx.x >> 5) : 0;
    dep_wait();   // the work counter, sweep numbers and spins of the step before
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
            if (threadIdx.x < 32) sthr[threadIdx.x] = threadIdx.x < 16 ? sg.thr16[threadIdx.x] : 0xFFFFFFFFu;
            loaded = (int)w.x;
            __syncthreads();
        }
        const SweepView v = sweep_view(sg);
        Counts cnt;
        batch_any_item<kColour, kNE, kAligned, kCMode>(v, sthr, w.y, passes, gtab[warp], dq[warp], cnt);
        if constexpr (kColour == 1) flush(v, v.ctrl->sweep, cnt, kNE, red);   // ends with __syncthreads()
        __syncthreads();
    }
    dep_launch();   // no items left: the next kernel may be scheduled
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
                wide_chunk<kNE, W, true>(v, sthr, 0, sweep, pp, y1, k1, cnt, u0);
            }
            __syncthreads();
            if (act) wide_chunk<kNE, W, true>(v, sthr, 1, sweep, pp, y1, k1, cnt, u1);
        } else {
            for (uint32_t t = threadIdx.x; t < total; t += blockDim.x)
                wide_chunk<kNE, W>(v, sthr, 0, sweep, pp, (int)(t / cpr), (int)(t % cpr), cnt);
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < total; t += blockDim.x)
                wide_chunk<kNE, W>(v, sthr, 1, sweep, pp, (int)(t / cpr), (int)(t % cpr), cnt);
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

bool any_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && g.cpl == nullptr && (g.L % 2) == 0)) return false;
    if (g.model == LAT_POTTS) return false;
    for (int k = 0; k < 16; ++k) {
        if ((k & 7) > 4) continue;
        if (!((g.always16 >> k) & 1u) && g.thr16[k] == 0u) return false;
    }
    return true;
}

int any_items(const Geom &g, int passes)
{
    const AnyItemShape sh = any_item_shape(g.half, (uint32_t)passes);
    return (int)((((uint32_t)g.L + sh.br - 1u) / sh.br) * sh.nseg);
}

int batch_any_grid(bool ne)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ne) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_any<true, false, 1>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_any<false, false, 1>, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_any(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item, int colour,
                             bool ne, bool cmode, bool aligned, int passes, int grid, cudaStream_t st)
{
    using K = void (*)(const Geom *, const uint2 *, int, unsigned *, uint32_t);
    // [Ising, North-East at T, North-East in c-mode][aligned][colour]
    static const K kern[3][2][2] = {
        {{k_batch_any<false, false, 0>, k_batch_any<false, false, 1>},
         {k_batch_any<false, true, 0>, k_batch_any<false, true, 1>}},
        {{k_batch_any<true, false, 0>, k_batch_any<true, false, 1>},
         {k_batch_any<true, true, 0>, k_batch_any<true, true, 1>}},
        {{k_batch_any<true, false, 0, true>, k_batch_any<true, false, 1, true>},
         {k_batch_any<true, true, 0, true>, k_batch_any<true, true, 1, true>}}};
    const int m = ne ? (cmode ? 2 : 1) : 0;
    return launch_pdl(kern[m][aligned ? 1 : 0][colour ? 1 : 0], (unsigned)grid, kThreads, st, geoms, items, n_items,
                      next_item, (uint32_t)passes);
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
    if (!wide_supported(g)) {   // L % 32 != 0: the any-L kernels, 16 sites per lane
        static int res_any = 0;
        const uint64_t chunks = (uint64_t)g.L * ((g.half + 15u) >> 4);
        const unsigned gb = (unsigned)std::min<long long>(
            (long long)((chunks + kThreads - 1) / kThreads),
            wave(reinterpret_cast<const void *>(k_any_pipe_ne<1, true>), res_any));
        using KG = void (*)(Geom, int);
        const bool ne = g.model == LAT_NE, ref = k.ref != nullptr;
        // North-East: [c-mode][reference][colour]
        static const KG kne[2][2][2] = {
            {{k_any_pipe_ne<0, false>, k_any_pipe_ne<1, false>}, {k_any_pipe_ne<0, true>, k_any_pipe_ne<1, true>}},
            {{k_any_pipe_ne<0, false, true>, k_any_pipe_ne<1, false, true>},
             {k_any_pipe_ne<0, true, true>, k_any_pipe_ne<1, true, true>}}};
        const int cm = g.cmode ? 1 : 0;
        const KG c0 = ne ? kne[cm][ref][0] : (ref ? k_any_pipe<0, true> : k_any_pipe<0, false>);
        const KG c1 = ne ? kne[cm][ref][1] : (ref ? k_any_pipe<1, true> : k_any_pipe<1, false>);
        cudaError_t e = launch_pdl(c0, gb, kThreads, st, k, off);
        return e == cudaSuccess ? launch_pdl(c1, gb, kThreads, st, k, off) : e;
    }
    if (g.model == LAT_NE && g.cpl == nullptr) {   // North-East: pipelined, draws compacted per warp
        static int res_ne = 0;
        const unsigned pb = (unsigned)std::min<long long>(
            wide_chunks(g), wave(reinterpret_cast<const void *>(k_wide_pipe_ne<1, true>), res_ne));
        using KG = void (*)(Geom, int);
        static const KG kne[2][2][2] = {
            {{k_wide_pipe_ne<0, false>, k_wide_pipe_ne<1, false>}, {k_wide_pipe_ne<0, true>, k_wide_pipe_ne<1, true>}},
            {{k_wide_pipe_ne<0, false, true>, k_wide_pipe_ne<1, false, true>},
             {k_wide_pipe_ne<0, true, true>, k_wide_pipe_ne<1, true, true>}}};
        const int cm = g.cmode ? 1 : 0, ref = k.ref != nullptr ? 1 : 0;
        cudaError_t e = launch_pdl(kne[cm][ref][0], pb, kThreads, st, k, off);
        return e == cudaSuccess ? launch_pdl(kne[cm][ref][1], pb, kThreads, st, k, off) : e;
    }
    // Ising, uniform or with per-bond couplings (and per-site field signs):
    // the software-pipelined kernels
    using KP = void (*)(Geom, int);
    static const KP pipe[3][2][2] = {
        {{k_wide_pipe<0, false>, k_wide_pipe<1, false>}, {k_wide_pipe<0, true>, k_wide_pipe<1, true>}},
        {{k_wide_pipe<0, false, true, false>, k_wide_pipe<1, false, true, false>},
         {k_wide_pipe<0, true, true, false>, k_wide_pipe<1, true, true, false>}},
        {{k_wide_pipe<0, false, true, true>, k_wide_pipe<1, false, true, true>},
         {k_wide_pipe<0, true, true, true>, k_wide_pipe<1, true, true, true>}}};
    static int res_pipe[3] = {0, 0, 0};
    const int m = g.cpl == nullptr ? 0 : (fields ? 2 : 1);
    const int ref = k.ref != nullptr ? 1 : 0;
    const unsigned pb = (unsigned)std::min<long long>(
        wide_chunks(g), wave(reinterpret_cast<const void *>(pipe[m][1][1]), res_pipe[m]));
    for (int colour = 0; colour < 2; ++colour) {
        cudaError_t e = launch_pdl(pipe[m][ref][colour], pb, kThreads, st, k, off);
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


}  // namespace lat
