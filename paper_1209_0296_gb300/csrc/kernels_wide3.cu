// kernels_wide3.cu -- two launches per sweep (one per colour, the kernel
// boundary being the device-wide barrier of §III.A steps 6-7) for Ising
// lattices that are 3D or have spin S > 1/2 (the extension of §III: "any
// spin value"), int8 spins in the checkerboard-planar layout, L a multiple
// of 16.
//
// A thread owns 8 consecutive same-colour sites of one plane row (one 8-byte
// load).  Neighbour sums of the 8 sites come from byte-wise additions: each
// neighbour byte is first offset by smax (so every byte is in [0, 2 smax])
// with a carry-free SWAR add, then the 2*dims neighbour words are summed
// with plain adds (at most 6 * 2 * 8 = 96 per byte, no carries).  The
// proposal, dE index, table lookup and acceptance follow the generic
// kernel site by site; draws come from the same Philox groups (4 sites per
// call for spin-1/2, 2 for spin-S).  The solo kernel reads s[sweep & 1]
// and writes s[(sweep+1) & 1] without copying a plane (colour 1 takes the
// new colour-0 sites from the new buffer); the batched kernel copies the
// colour-1 plane at colour 0 and updates it in place.  Colour 1 reduces the
// sweep's counters.
#include <algorithm>

#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxTab = 2465;  // largest table: two_S = 7, 3D

// Byte-wise a + b for bytes whose true sums stay in [0, 255] (no carry
// between bytes).
LAT_D uint32_t add_bytes(uint32_t a, uint32_t b)
{
    return ((a & 0x7F7F7F7Fu) + (b & 0x7F7F7F7Fu)) ^ ((a ^ b) & 0x80808080u);
}

// Per-thread partial sums.  32 bits suffice: a thread sees at most
// 2^32 / (resident threads) sites (< 2^17), each adding at most 6*S*S <= 96
// to |bond|.
struct Acc3 {
    int bond = 0, mag = 0, up = 0, acf = 0;
};

// The fields of a Geom that this kernel reads, small enough for registers.
struct View3 {
    int dims, L, two_S, dsmax, nmax, nn;
    uint32_t G, rows, half;
    uint64_t plane;
    int8_t *s0, *s1;
    const int8_t *ref;
};

LAT_D View3 view3(const Geom &g)
{
    View3 v;
    v.dims = g.dims;
    v.L = g.L;
    v.two_S = g.two_S;
    v.dsmax = g.dsmax;
    v.nmax = g.nmax;
    v.nn = g.nn;
    v.G = g.G;
    v.rows = g.rows;
    v.half = g.half;
    v.plane = g.plane;
    v.s0 = g.s[0];
    v.s1 = g.s[1];
    v.ref = g.ref;
    return v;
}

// Colour `colour` of the 8-site chunk k of plane row r = y + L*z.  TS and
// D fix two_S and dims at compile time (0: read them from g), which turns
// the spin/state maps, the proposal and the table index into constants.
template <int SH, int TS, int D>
LAT_D void wide3_chunk(const View3 &g, const TabEntry *stab, int colour, unsigned long long sweep,
                       const PhiloxPre &pp, uint32_t r, uint32_t k, Acc3 &acc)
{
    const int two_S = TS ? TS : g.two_S;
    const int dims = D ? D : g.dims;
    const int dsmax = TS ? 2 * max_spin(TS) : g.dsmax;
    const int nmax = (TS && D) ? 2 * D * max_spin(TS) : g.nmax;
    const int nn = (TS && D) ? 2 * nmax + 1 : g.nn;
    const int8_t *src = (sweep & 1) ? g.s1 : g.s0;
    int8_t *dst = (sweep & 1) ? g.s0 : g.s1;
    if (colour == 1) src = dst;
    const int L = g.L;
    const uint32_t half = g.half;
    const int oc = 1 - colour;
    const int y = (int)(r % (uint32_t)L), z = (int)(r / (uint32_t)L);
    auto row = [&](int c, uint32_t rr) { return src + (uint64_t)c * g.plane + (uint64_t)rr * half; };
    const uint32_t ym = (uint32_t)((y == 0 ? L - 1 : y - 1) + L * z);
    const uint32_t yp = (uint32_t)((y == L - 1 ? 0 : y + 1) + L * z);
    const uint2 S = *reinterpret_cast<const uint2 *>(row(colour, r) + 8 * k);
    const uint2 O = *reinterpret_cast<const uint2 *>(row(oc, r) + 8 * k);
    const uint2 Yn = *reinterpret_cast<const uint2 *>(row(oc, ym) + 8 * k);
    const uint2 Ys = *reinterpret_cast<const uint2 *>(row(oc, yp) + 8 * k);
    uint2 Zd = make_uint2(0u, 0u), Zu = make_uint2(0u, 0u);
    if (dims == 3) {
        const uint32_t zm = (uint32_t)(y + L * (z == 0 ? L - 1 : z - 1));
        const uint32_t zp = (uint32_t)(y + L * (z == L - 1 ? 0 : z + 1));
        Zd = *reinterpret_cast<const uint2 *>(row(oc, zm) + 8 * k);
        Zu = *reinterpret_cast<const uint2 *>(row(oc, zp) + 8 * k);
    }
    // draws first: they do not depend on the loads in flight
    const uint32_t g0 = r * g.G + ((8u * k) >> SH);  // first Philox group of the chunk
    constexpr int kCalls = 8 >> SH;
    U4 u[kCalls];
#pragma unroll
    for (int c = 0; c < kCalls; ++c) u[c] = philox_item(pp, g0 + (uint32_t)c, (uint32_t)colour);
    // row-shifted neighbours: x = 2j + p with p = (colour + y + z) & 1
    const bool p1 = ((colour + y + z) & 1) != 0;
    const uint32_t nwr = half >> 2;
    uint2 Lf, R;
    if (!p1) {  // west is j-1 of the other plane, east is j
        const uint32_t prev = reinterpret_cast<const uint32_t *>(row(oc, r))[wrap_once(2 * k - 1 + nwr, nwr)];
        Lf.x = __funnelshift_l(prev, O.x, 8);
        Lf.y = __funnelshift_l(O.x, O.y, 8);
        R = O;
    } else {    // west is j, east is j+1
        const uint32_t next = reinterpret_cast<const uint32_t *>(row(oc, r))[wrap_once(2 * k + 2, nwr)];
        Lf = O;
        R.x = __funnelshift_r(O.x, O.y, 8);
        R.y = __funnelshift_r(O.y, next, 8);
    }
    // neighbour sums offset by 2*dims*smax, byte-wise
    const int smax = max_spin(two_S);
    const uint32_t off = 0x01010101u * (uint32_t)smax;
    uint32_t nlo = add_bytes(Lf.x, off) + add_bytes(R.x, off) + add_bytes(Yn.x, off) + add_bytes(Ys.x, off);
    uint32_t nhi = add_bytes(Lf.y, off) + add_bytes(R.y, off) + add_bytes(Yn.y, off) + add_bytes(Ys.y, off);
    if (dims == 3) {
        nlo += add_bytes(Zd.x, off) + add_bytes(Zu.x, off);
        nhi += add_bytes(Zd.y, off) + add_bytes(Zu.y, off);
    }
    const int noff = 2 * dims * smax;
    uint32_t out_lo = 0, out_hi = 0;
    uint2 RS = make_uint2(0u, 0u), RO = RS;   // reference words (colour 1 only)
    const bool has_ref = colour == 1 && g.ref != nullptr;
    if (has_ref) {
        RS = *reinterpret_cast<const uint2 *>(g.ref + g.plane + (uint64_t)r * half + 8 * k);
        RO = *reinterpret_cast<const uint2 *>(g.ref + (uint64_t)r * half + 8 * k);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t sw = q < 4 ? S.x : S.y, nw = q < 4 ? nlo : nhi, ow = q < 4 ? O.x : O.y;
        const int sh8 = 8 * (q & 3);
        const int s_old = (int)(int8_t)(sw >> sh8);
        const int n = (int)((nw >> sh8) & 0xFFu) - noff;
        int s_new;
        uint32_t u_acc;
        if (SH == 2) {
            s_new = -s_old;   // spin-1/2: the flip
            u_acc = word_of(u[q >> 2], q & 3);
        } else {
            const int w = 2 * (q & 1);
            u_acc = word_of(u[q >> 1], w);
            const uint32_t u_prop = word_of(u[q >> 1], w + 1);
            const int k_old = state_of_spin(two_S, s_old);
            int k_new = k_old + 1 + (int)(((uint64_t)u_prop * (uint64_t)two_S) >> 32);
            if (k_new > two_S) k_new -= two_S + 1;
            s_new = spin_of_state(two_S, k_new);
        }
        const TabEntry e = stab[(s_new - s_old + dsmax) * nn + (n + nmax)];
        const int s_fin = (e.always || u_acc < e.thr) ? s_new : s_old;
        const uint32_t b = ((uint32_t)s_fin & 0xFFu) << sh8;
        if (q < 4) out_lo |= b;
        else out_hi |= b;
        if (colour == 1) {
            const int so = (int)(int8_t)(ow >> sh8);
            acc.bond += s_fin * n;
            acc.mag += s_fin + so;
            acc.up += (s_fin > 0) + (so > 0);
            if (has_ref) {
                const int rs = (int)(int8_t)((q < 4 ? RS.x : RS.y) >> sh8);
                const int ro = (int)(int8_t)((q < 4 ? RO.x : RO.y) >> sh8);
                acc.acf += s_fin * rs + so * ro;
            }
        }
    }
    *reinterpret_cast<uint2 *>(dst + (uint64_t)colour * g.plane + (uint64_t)r * half + 8 * k) =
        make_uint2(out_lo, out_hi);
    if (colour == 0) *reinterpret_cast<uint2 *>(dst + g.plane + (uint64_t)r * half + 8 * k) = O;
}

// ---------------------------------------------------------------------
// Software-pipelined solo form: each thread walks one 8-site chunk column
// down the plane rows r = y + L*z (rs rows apart) with two chunks in
// flight, the loads and Philox draws of the next chunk in the same block as
// the Metropolis step of this one (the draws load the FMA pipe, the step
// the ALU pipe).  Colour 0 reads both planes of the old buffer and writes
// plane 0 of the new one; colour 1 reads its own old sites from the old
// buffer and the new colour-0 sites from the new one, and writes plane 1:
// no plane is copied.  Same chunks, draws and bits as wide3_chunk.
// ---------------------------------------------------------------------
struct W3In {
    uint2 S, O, Yn, Ys, Zd, Zu;
    uint32_t nb;   // the other plane's word past the chunk (west word for x = 2j, east word for x = 2j+1)
};

template <int D>
struct W3Walk {
    const int8_t *pS, *pO;   // this colour's old sites, the other colour's current sites (plane bases)
    int8_t *dS;              // this colour's plane in the new buffer
    const int8_t *r1, *r0;   // reference planes 1 and 0 (or null)
    uint32_t half, L, G, k, nwr;
    uint32_t wprev, wnext;   // word index in the row of the west word (p = 0) / east word (p = 1)
};

template <int kColour>
LAT_D void w3_load(const View3 &g, const int8_t *pS, const int8_t *pO, uint32_t half, uint32_t L, int dims,
                   uint32_t r, uint32_t y, uint32_t z, uint32_t k, uint32_t wprev, uint32_t wnext, W3In &in)
{
    const uint32_t ym = (y == 0 ? L - 1 : y - 1) + L * z;
    const uint32_t yp = (y == L - 1 ? 0 : y + 1) + L * z;
    in.S = *reinterpret_cast<const uint2 *>(pS + (size_t)r * half + 8 * k);
    in.O = *reinterpret_cast<const uint2 *>(pO + (size_t)r * half + 8 * k);
    in.Yn = *reinterpret_cast<const uint2 *>(pO + (size_t)ym * half + 8 * k);
    in.Ys = *reinterpret_cast<const uint2 *>(pO + (size_t)yp * half + 8 * k);
    in.Zd = make_uint2(0u, 0u);
    in.Zu = make_uint2(0u, 0u);
    if (dims == 3) {
        const uint32_t zm = y + L * (z == 0 ? L - 1 : z - 1);
        const uint32_t zp = y + L * (z == L - 1 ? 0 : z + 1);
        in.Zd = *reinterpret_cast<const uint2 *>(pO + (size_t)zm * half + 8 * k);
        in.Zu = *reinterpret_cast<const uint2 *>(pO + (size_t)zp * half + 8 * k);
    }
    const bool p1 = ((kColour + y + z) & 1) != 0;
    in.nb = reinterpret_cast<const uint32_t *>(pO + (size_t)r * half)[p1 ? wnext : wprev];
}

template <int SH, int TS, int D, int kColour, bool kRef>
LAT_D void w3_step(const View3 &g, const TabEntry *stab, int8_t *dS, const int8_t *r1, const int8_t *r0, uint32_t r,
                   uint32_t y, uint32_t z, uint32_t k, const W3In &in, const U4 (&u)[8 >> SH], Acc3 &acc)
{
    const int two_S = TS ? TS : g.two_S;
    const int dims = D ? D : g.dims;
    const int dsmax = TS ? 2 * max_spin(TS) : g.dsmax;
    const int nmax = (TS && D) ? 2 * D * max_spin(TS) : g.nmax;
    const int nn = (TS && D) ? 2 * nmax + 1 : g.nn;
    const uint32_t half = g.half;
    const bool p1 = ((kColour + y + z) & 1) != 0;
    uint2 Lf, R;
    if (!p1) {   // west is j-1 of the other plane, east is j
        Lf.x = __funnelshift_l(in.nb, in.O.x, 8);
        Lf.y = __funnelshift_l(in.O.x, in.O.y, 8);
        R = in.O;
    } else {     // west is j, east is j+1
        Lf = in.O;
        R.x = __funnelshift_r(in.O.x, in.O.y, 8);
        R.y = __funnelshift_r(in.O.y, in.nb, 8);
    }
    const int smax = max_spin(two_S);
    const uint32_t offb = 0x01010101u * (uint32_t)smax;
    uint32_t nlo = add_bytes(Lf.x, offb) + add_bytes(R.x, offb) + add_bytes(in.Yn.x, offb) + add_bytes(in.Ys.x, offb);
    uint32_t nhi = add_bytes(Lf.y, offb) + add_bytes(R.y, offb) + add_bytes(in.Yn.y, offb) + add_bytes(in.Ys.y, offb);
    if (dims == 3) {
        nlo += add_bytes(in.Zd.x, offb) + add_bytes(in.Zu.x, offb);
        nhi += add_bytes(in.Zd.y, offb) + add_bytes(in.Zu.y, offb);
    }
    const int noff = 2 * dims * smax;
    uint32_t out_lo = 0, out_hi = 0;
    uint2 RS = make_uint2(0u, 0u), RO = RS;
    if constexpr (kColour == 1 && kRef) {
        RS = *reinterpret_cast<const uint2 *>(r1 + (size_t)r * half + 8 * k);
        RO = *reinterpret_cast<const uint2 *>(r0 + (size_t)r * half + 8 * k);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t sw = q < 4 ? in.S.x : in.S.y, nw = q < 4 ? nlo : nhi, ow = q < 4 ? in.O.x : in.O.y;
        const int sh8 = 8 * (q & 3);
        const int s_old = (int)(int8_t)(sw >> sh8);
        const int n = (int)((nw >> sh8) & 0xFFu) - noff;
        int s_new;
        uint32_t u_acc;
        if (SH == 2) {
            s_new = -s_old;
            u_acc = word_of(u[q >> 2], q & 3);
        } else {
            const int w = 2 * (q & 1);
            u_acc = word_of(u[q >> 1], w);
            const uint32_t u_prop = word_of(u[q >> 1], w + 1);
            const int k_old = state_of_spin(two_S, s_old);
            int k_new = k_old + 1 + (int)(((uint64_t)u_prop * (uint64_t)two_S) >> 32);
            if (k_new > two_S) k_new -= two_S + 1;
            s_new = spin_of_state(two_S, k_new);
        }
        const TabEntry e = stab[(s_new - s_old + dsmax) * nn + (n + nmax)];
        const int s_fin = (e.always || u_acc < e.thr) ? s_new : s_old;
        const uint32_t b = ((uint32_t)s_fin & 0xFFu) << sh8;
        if (q < 4) out_lo |= b;
        else out_hi |= b;
        if constexpr (kColour == 1) {
            const int so = (int)(int8_t)(ow >> sh8);
            acc.bond += s_fin * n;
            acc.mag += s_fin + so;
            acc.up += (s_fin > 0) + (so > 0);
            if constexpr (kRef) {
                const int rs = (int)(int8_t)((q < 4 ? RS.x : RS.y) >> sh8);
                const int ro = (int)(int8_t)((q < 4 ? RO.x : RO.y) >> sh8);
                acc.acf += s_fin * rs + so * ro;
            }
        }
    }
    *reinterpret_cast<uint2 *>(dS + (size_t)r * half + 8 * k) = make_uint2(out_lo, out_hi);
}

template <int SH, int TS, int D, int kColour, bool kRef>
__global__ void __launch_bounds__(kThreads, 2) k_wide3_pipe(Geom g, int off)
{
    __shared__ TabEntry stab[kMaxTab];
    __shared__ long long red[kThreads / 32];
    for (int i = threadIdx.x; i < g.tab_n; i += blockDim.x) stab[i] = g.tab[i];
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const View3 v = view3(g);
    const int dims = D ? D : v.dims;
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    const uint32_t plane = (uint32_t)v.plane;
    const int8_t *pS = old + (size_t)kColour * plane;
    const int8_t *pO = (kColour == 0 ? old : nw) + (size_t)(1 - kColour) * plane;
    int8_t *dS = nw + (size_t)kColour * plane;
    const int8_t *r1 = v.ref ? v.ref + plane : nullptr, *r0 = v.ref;
    Acc3 acc;
    const uint32_t cpr = v.half >> 3;   // 8-site chunks per plane row
    const uint32_t rows = v.rows, L = (uint32_t)v.L;
    const uint32_t rs = (gridDim.x * blockDim.x) / cpr;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t r = gt / cpr;
    const uint32_t k = gt - r * cpr;
    if (r < rs && r < rows) {
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        const uint32_t nwr = v.half >> 2;
        const uint32_t wprev = wrap_once(2 * k - 1 + nwr, nwr), wnext = wrap_once(2 * k + 2, nwr);
        // (y, z) of row r, stepped by rs rows without a division
        uint32_t y = r % L, z = r / L;
        const uint32_t dy = rs % L, dz = rs / L;
        auto step_row = [&](uint32_t &yy, uint32_t &zz) {
            yy += dy;
            zz += dz;
            if (yy >= L) {
                yy -= L;
                ++zz;
            }
        };
        constexpr int kCalls = 8 >> SH;
        auto draws = [&](uint32_t rr, U4 (&u)[kCalls]) {
            const uint32_t g0 = rr * v.G + ((8u * k) >> SH);
#pragma unroll
            for (int c = 0; c < kCalls; ++c) u[c] = philox_item(pp, g0 + (uint32_t)c, (uint32_t)kColour);
        };
        W3In A, B;
        U4 uA[kCalls], uB[kCalls];
        w3_load<kColour>(v, pS, pO, v.half, L, dims, r, y, z, k, wprev, wnext, A);
        draws(r, uA);
        for (;;) {
            const uint32_t r1_ = r + rs;
            uint32_t y1 = y, z1 = z;
            step_row(y1, z1);
            if (r1_ >= rows) {
                w3_step<SH, TS, D, kColour, kRef>(v, stab, dS, r1, r0, r, y, z, k, A, uA, acc);
                break;
            }
            w3_load<kColour>(v, pS, pO, v.half, L, dims, r1_, y1, z1, k, wprev, wnext, B);
            draws(r1_, uB);
            w3_step<SH, TS, D, kColour, kRef>(v, stab, dS, r1, r0, r, y, z, k, A, uA, acc);
            const uint32_t r2 = r1_ + rs;
            uint32_t y2 = y1, z2 = z1;
            step_row(y2, z2);
            if (r2 >= rows) {
                w3_step<SH, TS, D, kColour, kRef>(v, stab, dS, r1, r0, r1_, y1, z1, k, B, uB, acc);
                break;
            }
            w3_load<kColour>(v, pS, pO, v.half, L, dims, r2, y2, z2, k, wprev, wnext, A);
            draws(r2, uA);
            w3_step<SH, TS, D, kColour, kRef>(v, stab, dS, r1, r0, r1_, y1, z1, k, B, uB, acc);
            r = r2;
            y = y2;
            z = z2;
        }
    }
    if constexpr (kColour == 1) {
        unsigned long long *slot = series_slot(g.ctrl, sweep);
        long long t;
        t = block_sum_ll((long long)acc.bond, red);
        if (threadIdx.x == 0) add_counter(slot + 0, t);
        t = block_sum_ll((long long)acc.mag, red);
        if (threadIdx.x == 0) add_counter(slot + 1, t);
        t = block_sum_ll((long long)acc.up, red);
        if (threadIdx.x == 0) add_counter(slot + 2, t);
        if constexpr (kRef) {
            t = block_sum_ll((long long)acc.acf, red);
            if (threadIdx.x == 0) add_counter(acf_slot(g.ctrl, sweep), t);
        }
    }
}

// Batched form: a persistent grid takes (lattice, item) pairs from an
// atomic counter; an item is kItemChunks x kThreads chunks of one colour of
// one lattice.  The lattice's descriptor and table are reloaded only when a
// CTA moves to another lattice (items are ordered by lattice).
constexpr int kItemChunks = 4;

__global__ void __launch_bounds__(kThreads, 4) k_batch_wide3(const Geom *geoms, const uint2 *items, int n_items,
                                                         unsigned *next_item, int colour)
{
    __shared__ TabEntry stab[kMaxTab];
    __shared__ long long red[kThreads / 32];
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
            for (int i = threadIdx.x; i < sg.tab_n; i += blockDim.x) stab[i] = sg.tab[i];
            loaded = (int)w.x;
            __syncthreads();
        }
        // register copies: no aliasing with shared-memory stores
        const View3 g = view3(sg);
        Ctrl *const ctrl = sg.ctrl;
        const bool spin_half = sg.sh == 2;   // wide3 takes 2D spin-1/2 never, so this is 3D
        const bool spin_one3 = sg.two_S == 2 && sg.dims == 3;
        const unsigned long long sweep = ctrl->sweep;
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), sg.key0, sg.key1);
        const uint32_t cpr = g.half >> 3;
        const uint32_t total = g.rows * cpr;   // < 2^28 (N < 2^32)
        Acc3 acc;
#pragma unroll 1
        for (int c = 0; c < kItemChunks; ++c) {
            const uint32_t t = (w.y * (uint32_t)kItemChunks + (uint32_t)c) * kThreads + threadIdx.x;
            if (t >= total) break;
            const uint32_t rr = t / cpr, kk = t - rr * cpr;
            if (spin_half) wide3_chunk<2, 1, 3>(g, stab, colour, sweep, pp, rr, kk, acc);
            else if (spin_one3) wide3_chunk<1, 2, 3>(g, stab, colour, sweep, pp, rr, kk, acc);
            else wide3_chunk<1, 0, 0>(g, stab, colour, sweep, pp, rr, kk, acc);
        }
        if (colour == 1) {
            unsigned long long *slot = series_slot(ctrl, sweep);
            long long v;
            v = block_sum_ll((long long)acc.bond, red);
            if (threadIdx.x == 0) add_counter(slot + 0, v);
            v = block_sum_ll((long long)acc.mag, red);
            if (threadIdx.x == 0) add_counter(slot + 1, v);
            v = block_sum_ll((long long)acc.up, red);
            if (threadIdx.x == 0) add_counter(slot + 2, v);
            if (g.ref != nullptr) {
                v = block_sum_ll((long long)acc.acf, red);
                if (threadIdx.x == 0) add_counter(acf_slot(ctrl, sweep), v);
            }
        }
        __syncthreads();
    }
}

}  // namespace

int wide3_items(const Geom &g)
{
    const uint64_t chunks = (uint64_t)g.rows * (g.half >> 3);
    const uint64_t per = (uint64_t)kItemChunks * kThreads;
    return (int)((chunks + per - 1) / per);
}

int batch_wide3_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_wide3, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_wide3(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int colour, int grid, cudaStream_t st)
{
    k_batch_wide3<<<grid, kThreads, 0, st>>>(geoms, items, n_items, next_item, colour);
    return cudaGetLastError();
}

bool wide3_supported(const Geom &g)
{
    return g.model == LAT_ISING && (g.dims == 3 || g.two_S >= 2) && (g.L % 16) == 0 &&
           g.bits[0] == nullptr && g.cpl == nullptr && g.tab_n <= kMaxTab;
}

cudaError_t launch_sweep_wide3(const Geom &g, int off, cudaStream_t st)
{
    // instantiations: 3D spin-1/2, 3D spin-1, 2D spin-1, any other spin-S;
    // each colour, with and without a reference state
    const int which = g.two_S == 1 ? 0 : (g.two_S == 2 ? (g.dims == 3 ? 1 : 2) : 3);
    const int ref = g.ref != nullptr ? 1 : 0;
    using K = void (*)(Geom, int);
    static const K kern[4][2][2] = {
        {{k_wide3_pipe<2, 1, 3, 0, false>, k_wide3_pipe<2, 1, 3, 1, false>},
         {k_wide3_pipe<2, 1, 3, 0, true>, k_wide3_pipe<2, 1, 3, 1, true>}},
        {{k_wide3_pipe<1, 2, 3, 0, false>, k_wide3_pipe<1, 2, 3, 1, false>},
         {k_wide3_pipe<1, 2, 3, 0, true>, k_wide3_pipe<1, 2, 3, 1, true>}},
        {{k_wide3_pipe<1, 2, 2, 0, false>, k_wide3_pipe<1, 2, 2, 1, false>},
         {k_wide3_pipe<1, 2, 2, 0, true>, k_wide3_pipe<1, 2, 2, 1, true>}},
        {{k_wide3_pipe<1, 0, 0, 0, false>, k_wide3_pipe<1, 0, 0, 1, false>},
         {k_wide3_pipe<1, 0, 0, 0, true>, k_wide3_pipe<1, 0, 0, 1, true>}}};
    static int resident[4] = {0, 0, 0, 0};
    if (resident[which] == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern[which][1][1], kThreads, 0);
        resident[which] = sms * (per > 0 ? per : 1);
    }
    const uint64_t chunks = (uint64_t)g.rows * (g.half >> 3);
    const unsigned blocks = (unsigned)std::min<uint64_t>((chunks + kThreads - 1) / kThreads,
                                                        (uint64_t)resident[which]);
    for (int colour = 0; colour < 2; ++colour) {
        kern[which][ref][colour]<<<blocks, kThreads, 0, st>>>(g, off);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lat
