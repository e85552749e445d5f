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
// call for spin-1/2, 2 for spin-S).  The kernels (solo and batched) read
// s[sweep & 1] and write s[(sweep+1) & 1] without copying a plane (colour 1
// takes the new colour-0 sites from the new buffer).  Colour 1 reduces the
// sweep's counters.  Spin-1/2 and spin-1 lattices whose tables hold no
// never-accept entry take a byte-parallel step (four sites per word).
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

// ---------------------------------------------------------------------
// Software-pipelined solo form: each thread walks one 8-site chunk column
// down the plane rows r = y + L*z (rs rows apart) with two chunks in
// flight, the loads and Philox draws of the next chunk in the same block as
// the Metropolis step of this one (the draws load the FMA pipe, the step
// the ALU pipe).  Colour 0 reads both planes of the old buffer and writes
// plane 0 of the new one; colour 1 reads its own old sites from the old
// buffer and the new colour-0 sites from the new one, and writes plane 1:
// no plane is copied.  Same chunks and draws as the generic kernel.
// ---------------------------------------------------------------------
struct W3In {
    uint2 S, O, Yn, Ys, Zd, Zu;
    uint32_t nb;   // the other plane's word past the chunk (west word for x = 2j, east word for x = 2j+1)
    uint32_t o;    // byte offset of the chunk in its plane: r * half + 8k
};

// Per-thread constants of the column walk: byte offsets within a plane
// (N < 2^32, so a plane is below 2^31 bytes and 32-bit offsets suffice).
struct W3Geo {
    uint32_t half, L, k8;
    uint32_t wrap_y;   // (L - 1) * half: from row y = 0 to y = L - 1
    uint32_t step_z;   // L * half: one z layer
    uint32_t wrap_z;   // (L - 1) * L * half: from z = 0 to z = L - 1
    uint32_t wp4, wn4; // byte offsets in a row of the west word (x = 2j) / east word (x = 2j + 1)
};

LAT_D W3Geo w3_geo(uint32_t half, uint32_t L, uint32_t k, uint32_t wprev, uint32_t wnext)
{
    W3Geo c;
    c.half = half;
    c.L = L;
    c.k8 = 8u * k;
    c.wrap_y = (L - 1u) * half;
    c.step_z = L * half;
    c.wrap_z = (L - 1u) * L * half;
    c.wp4 = 4u * wprev;
    c.wn4 = 4u * wnext;
    return c;
}

template <int kColour>
LAT_D void w3_load(const W3Geo &c, const int8_t *pS, const int8_t *pO, int dims, uint32_t r, uint32_t y, uint32_t z,
                   W3In &in)
{
    const uint32_t row = r * c.half, o = row + c.k8;
    const uint32_t oym = y == 0 ? o + c.wrap_y : o - c.half;
    const uint32_t oyp = y == c.L - 1u ? o - c.wrap_y : o + c.half;
    in.o = o;
    in.S = *reinterpret_cast<const uint2 *>(pS + o);
    in.O = *reinterpret_cast<const uint2 *>(pO + o);
    in.Yn = *reinterpret_cast<const uint2 *>(pO + oym);
    in.Ys = *reinterpret_cast<const uint2 *>(pO + oyp);
    in.Zd = make_uint2(0u, 0u);
    in.Zu = make_uint2(0u, 0u);
    if (dims == 3) {
        const uint32_t ozm = z == 0 ? o + c.wrap_z : o - c.step_z;
        const uint32_t ozp = z == c.L - 1u ? o - c.wrap_z : o + c.step_z;
        in.Zd = *reinterpret_cast<const uint2 *>(pO + ozm);
        in.Zu = *reinterpret_cast<const uint2 *>(pO + ozp);
    }
    const bool p1 = ((kColour + y + z) & 1) != 0;
    in.nb = *reinterpret_cast<const uint32_t *>(pO + row + (p1 ? c.wn4 : c.wp4));
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
        RS = *reinterpret_cast<const uint2 *>(r1 + in.o);
        RO = *reinterpret_cast<const uint2 *>(r0 + in.o);
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
    *reinterpret_cast<uint2 *>(dS + in.o) = make_uint2(out_lo, out_hi);
}

// ---------------------------------------------------------------------
// Byte-parallel step for spin-1/2 and spin-1 (TS = 1, 2): the proposal,
// the table index, the acceptance mask and the counters are formed for the
// four sites of a word at once; per site remain one byte extract, one
// table lookup and one compare.  Spins are bytes s in {-1, 0, 1} (0xFF,
// 0x00, 0x01); k = s + 1 is the state in {0, 1, 2} (spin-1/2: {0, 2}).
// The table is the compact form t'[r * nn + n + nmax] = (always ? ~0 :
// thr - 1), accept iff u <= t', with row r = 0, 1, 2, 3 for ds = s' - s =
// -2, -1, +1, +2; it needs a table without never-accept entries.
// ---------------------------------------------------------------------

// k = s + 1 byte-wise: the word add carries out of each 0xFF byte, and that
// carry is taken back from the byte above (the top byte's leaves the word).
LAT_D uint32_t plus_one_bytes(uint32_t v) { return v + 0x01010101u - ((v << 1) & 0x01010100u); }

// s = k - 1 byte-wise for k in {0, 1, 2}: the word subtract borrows from the
// byte above each zero byte, and that borrow is given back.
LAT_D uint32_t minus_one_bytes(uint32_t k)
{
    return k - 0x01010101u + ((~(k | (k >> 1)) & 0x01010101u) << 8);
}

LAT_D uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Byte q = bit 31 of word q: a selector nibble with bit 3 set copies the
// sign of the chosen byte (byte 3 of a word) over the whole target byte.
LAT_D uint32_t top_bits(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3)
{
    const uint32_t t01 = prmt(u0, u1, 0x00FBu), t23 = prmt(u2, u3, 0x00FBu);
    return prmt(t01, t23, 0x5410u) & 0x01010101u;
}

// 0xFF in each byte whose bit 7 is set, else 0x00.
LAT_D uint32_t sign_bytes(uint32_t x) { return prmt(x, 0u, 0xBA98u); }

constexpr int kSwarTab = 4 * 13;   // rows x nn, nn <= 13 (3D, nmax = 6)

// Rows of the compact table: ds = -2, -1, +1, +2.
LAT_HD int swar_ds(int row) { return row < 2 ? row - 2 : row - 1; }

template <int TS, int D, int kColour, bool kRef>
LAT_D void w3s_word(uint32_t S, uint32_t O, uint32_t nsum, uint32_t bits, const uint32_t *acc_u,
                    const char *tb, uint32_t &Sfin, Acc3 &acc, uint32_t R1, uint32_t R0)
{
    constexpr uint32_t ones = 0x01010101u;
    constexpr uint32_t nn4 = 4u * (2u * 2u * D + 1u);
    const uint32_t Ko = plus_one_bytes(S);
    uint32_t Kn;
    if constexpr (TS == 1) {
        Kn = 0x02020202u - Ko;                       // the flip: k' = 2 - k
    } else {
        Kn = Ko + ones + bits;                       // k + 1 + [u_prop >= 2^31], in [1, 4]
        Kn -= sign_bytes(Kn + 0x7D7D7D7Du) & 0x03030303u;   // wrap modulo 3 (bit 7 set iff k' >= 3)
    }
    const uint32_t X = Kn + 0x02020202u - Ko;        // ds + 2 in {0, 1, 3, 4}
    const uint32_t row = X - (((X + ones) >> 2) & ones);
    const uint32_t idx4 = row * nn4 + (nsum << 2);   // byte offsets, at most 204
    uint32_t am = 0;   // bit 7 of byte q: site q accepted
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t t = *reinterpret_cast<const uint32_t *>(tb + ((idx4 >> (8 * q)) & 0xFFu));
        am |= (acc_u[q] <= t ? 0x80u : 0u) << (8 * q);
    }
    const uint32_t m = sign_bytes(am);
    if constexpr (TS == 1) {
        Sfin = S ^ (m & 0xFEFEFEFEu);
    } else {
        Sfin = minus_one_bytes(Ko ^ ((Ko ^ Kn) & m));
    }
    if constexpr (kColour == 1) {
        // bond: sum s (n_sum - 2D), n_sum = n + 2D; up: (sum s + #nonzero) / 2
        const int ss = __dp4a((int)Sfin, (int)ones, 0), so = __dp4a((int)O, (int)ones, 0);
        acc.bond += __dp4a((int)Sfin, (int)nsum, 0) - 2 * D * ss;
        acc.mag += ss + so;
        const int nz = TS == 1 ? 8 : __popc(Sfin & ones) + __popc(O & ones);
        acc.up += (ss + so + nz) >> 1;
        if constexpr (kRef) acc.acf += __dp4a((int)Sfin, (int)R1, __dp4a((int)O, (int)R0, 0));
    }
}

template <int SH, int TS, int D, int kColour, bool kRef>
LAT_D void w3s_step(const View3 &g, const uint32_t *st4, int8_t *dS, const int8_t *r1, const int8_t *r0,
                    uint32_t r, uint32_t y, uint32_t z, uint32_t k, const W3In &in, const U4 (&u)[8 >> SH],
                    Acc3 &acc)
{
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
    // n + nmax = sum of the neighbours' k (each s + 1), at most 12 per byte
    uint32_t nlo = plus_one_bytes(Lf.x) + plus_one_bytes(R.x) + plus_one_bytes(in.Yn.x) + plus_one_bytes(in.Ys.x);
    uint32_t nhi = plus_one_bytes(Lf.y) + plus_one_bytes(R.y) + plus_one_bytes(in.Yn.y) + plus_one_bytes(in.Ys.y);
    if constexpr (D == 3) {
        nlo += plus_one_bytes(in.Zd.x) + plus_one_bytes(in.Zu.x);
        nhi += plus_one_bytes(in.Zd.y) + plus_one_bytes(in.Zu.y);
    }
    uint32_t ua_lo[4], ua_hi[4], b_lo = 0, b_hi = 0;
    if constexpr (TS == 1) {   // 4 sites per call: word q of call 0 (lo) and 1 (hi)
        ua_lo[0] = u[0].x, ua_lo[1] = u[0].y, ua_lo[2] = u[0].z, ua_lo[3] = u[0].w;
        ua_hi[0] = u[1].x, ua_hi[1] = u[1].y, ua_hi[2] = u[1].z, ua_hi[3] = u[1].w;
    } else {                   // 2 sites per call: acceptance words 0, 2, proposal words 1, 3
        ua_lo[0] = u[0].x, ua_lo[1] = u[0].z, ua_lo[2] = u[1].x, ua_lo[3] = u[1].z;
        ua_hi[0] = u[2].x, ua_hi[1] = u[2].z, ua_hi[2] = u[3].x, ua_hi[3] = u[3].z;
        b_lo = top_bits(u[0].y, u[0].w, u[1].y, u[1].w);
        b_hi = top_bits(u[2].y, u[2].w, u[3].y, u[3].w);
    }
    uint32_t R1lo = 0, R1hi = 0, R0lo = 0, R0hi = 0;
    if constexpr (kColour == 1 && kRef) {
        const uint2 RS = *reinterpret_cast<const uint2 *>(r1 + in.o);
        const uint2 RO = *reinterpret_cast<const uint2 *>(r0 + in.o);
        R1lo = RS.x, R1hi = RS.y, R0lo = RO.x, R0hi = RO.y;
    }
    const char *tb = reinterpret_cast<const char *>(st4);
    uint2 out;
    w3s_word<TS, D, kColour, kRef>(in.S.x, in.O.x, nlo, b_lo, ua_lo, tb, out.x, acc, R1lo, R0lo);
    w3s_word<TS, D, kColour, kRef>(in.S.y, in.O.y, nhi, b_hi, ua_hi, tb, out.y, acc, R1hi, R0hi);
    *reinterpret_cast<uint2 *>(dS + in.o) = out;
}

// kSwar: the byte-parallel step (TS = 1, 2 with a table free of
// never-accept entries), else the per-site one.
template <int SH, int TS, int D, int kColour, bool kRef, bool kSwar = false>
__global__ void __launch_bounds__(kThreads, 2) k_wide3_pipe(Geom g, int off)
{
    __shared__ TabEntry stab[kSwar ? 1 : kMaxTab];
    __shared__ uint32_t st4[kSwar ? kSwarTab : 1];
    __shared__ long long red[kThreads / 32];
    if constexpr (kSwar) {
        const int nn = g.nn;
        for (int i = threadIdx.x; i < 4 * nn; i += blockDim.x) {
            const int row = i / nn, col = i - row * nn;
            const TabEntry e = g.tab[(swar_ds(row) + g.dsmax) * nn + col];
            st4[i] = e.always ? 0xFFFFFFFFu : e.thr - 1u;
        }
    } else {
        for (int i = threadIdx.x; i < g.tab_n; i += blockDim.x) stab[i] = g.tab[i];
    }
    __syncthreads();
    dep_wait();
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
        const W3Geo geo = w3_geo(v.half, L, k, wrap_once(2 * k - 1 + nwr, nwr), wrap_once(2 * k + 2, nwr));
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
        auto step = [&](uint32_t rr, uint32_t yy, uint32_t zz, const W3In &in, const U4 (&u)[kCalls]) {
            if constexpr (kSwar) w3s_step<SH, TS, D, kColour, kRef>(v, st4, dS, r1, r0, rr, yy, zz, k, in, u, acc);
            else w3_step<SH, TS, D, kColour, kRef>(v, stab, dS, r1, r0, rr, yy, zz, k, in, u, acc);
        };
        W3In A, B;
        U4 uA[kCalls], uB[kCalls];
        w3_load<kColour>(geo, pS, pO, dims, r, y, z, A);
        draws(r, uA);
        for (;;) {
            const uint32_t r1_ = r + rs;
            uint32_t y1 = y, z1 = z;
            step_row(y1, z1);
            if (r1_ >= rows) {
                step(r, y, z, A, uA);
                break;
            }
            w3_load<kColour>(geo, pS, pO, dims, r1_, y1, z1, B);
            draws(r1_, uB);
            step(r, y, z, A, uA);
            const uint32_t r2 = r1_ + rs;
            uint32_t y2 = y1, z2 = z1;
            step_row(y2, z2);
            if (r2 >= rows) {
                step(r1_, y1, z1, B, uB);
                break;
            }
            w3_load<kColour>(geo, pS, pO, dims, r2, y2, z2, A);
            draws(r2, uA);
            step(r1_, y1, z1, B, uB);
            r = r2;
            y = y2;
            z = z2;
        }
    }
    dep_launch();   // main work done: the next kernel may be scheduled
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

// ---------------------------------------------------------------------
// Batched form: a persistent grid takes (lattice, item) pairs from an
// atomic counter.  An item is a band of plane rows x a segment of up to
// kThreads chunk columns of one colour of one lattice; each thread walks
// its column down the band (rsb rows apart) with two chunks in flight, as
// the solo kernel does, and the same no-copy convention.  The lattice's
// descriptor and table are reloaded only when a CTA moves to another
// lattice (items are ordered by lattice).  kSwar: the list of lattices that
// take the byte-parallel step (spin-1/2 and spin-1 with strict tables).
// ---------------------------------------------------------------------
template <int SH, int TS, int D, int kColour, bool kRef, bool kSwar>
LAT_D void batch_w3_item(const View3 &v, uint32_t key0, uint32_t key1, unsigned long long sweep,
                         const TabEntry *stab, const uint32_t *st4, uint32_t item, uint32_t passes, Acc3 &acc)
{
    const ColItemShape sh = col_item_shape(v.half, v.rows, passes);
    const uint32_t L = (uint32_t)v.L;
    const int dims = D ? D : v.dims;
    const uint32_t band = item / sh.nseg, seg = item - band * sh.nseg;
    const uint32_t r_end = min(v.rows, band * sh.br + sh.br);
    uint32_t k, r;
    if (sh.cpr <= (uint32_t)kThreads) {
        k = threadIdx.x % sh.cpr;
        r = band * sh.br + threadIdx.x / sh.cpr;
        if (threadIdx.x / sh.cpr >= sh.rsb) return;
    } else {
        k = seg * kThreads + threadIdx.x;
        r = band * sh.br;
        if (k >= sh.cpr) return;
    }
    if (r >= r_end) return;
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    const uint32_t plane = (uint32_t)v.plane;
    const int8_t *pS = old + (size_t)kColour * plane;
    const int8_t *pO = (kColour == 0 ? old : nw) + (size_t)(1 - kColour) * plane;
    int8_t *dS = nw + (size_t)kColour * plane;
    const int8_t *r1 = v.ref ? v.ref + plane : nullptr, *r0 = v.ref;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), key0, key1);
    const uint32_t nwr = v.half >> 2;
    const W3Geo geo = w3_geo(v.half, L, k, wrap_once(2 * k - 1 + nwr, nwr), wrap_once(2 * k + 2, nwr));
    uint32_t y = r % L, z = r / L;
    const uint32_t dy = sh.rsb % L, dz = sh.rsb / L;
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
    auto step = [&](uint32_t rr, uint32_t yy, uint32_t zz, const W3In &in, const U4 (&u)[kCalls]) {
        if constexpr (kSwar) w3s_step<SH, TS, D, kColour, kRef>(v, st4, dS, r1, r0, rr, yy, zz, k, in, u, acc);
        else w3_step<SH, TS, D, kColour, kRef>(v, stab, dS, r1, r0, rr, yy, zz, k, in, u, acc);
    };
    W3In A, B;
    U4 uA[kCalls], uB[kCalls];
    w3_load<kColour>(geo, pS, pO, dims, r, y, z, A);
    draws(r, uA);
    for (;;) {
        const uint32_t ra = r + sh.rsb;
        uint32_t ya = y, za = z;
        step_row(ya, za);
        if (ra >= r_end) {
            step(r, y, z, A, uA);
            break;
        }
        w3_load<kColour>(geo, pS, pO, dims, ra, ya, za, B);
        draws(ra, uB);
        step(r, y, z, A, uA);
        const uint32_t rb = ra + sh.rsb;
        uint32_t yb = ya, zb = za;
        step_row(yb, zb);
        if (rb >= r_end) {
            step(ra, ya, za, B, uB);
            break;
        }
        w3_load<kColour>(geo, pS, pO, dims, rb, yb, zb, A);
        draws(rb, uA);
        step(ra, ya, za, B, uB);
        r = rb;
        y = yb;
        z = zb;
    }
}

template <int kColour, bool kSwar>
__global__ void __launch_bounds__(kThreads, 2) k_batch_wide3(const Geom *geoms, const uint2 *items, int n_items,
                                                         unsigned *next_item, uint32_t passes)
{
    __shared__ TabEntry stab[kSwar ? 1 : kMaxTab];
    __shared__ uint32_t st4[kSwar ? kSwarTab : 1];
    __shared__ long long red[kThreads / 32];
    __shared__ Geom sg;
    __shared__ int cur;
    int loaded = -1;
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
            if constexpr (kSwar) {
                const int nn = sg.nn;
                for (int i = threadIdx.x; i < 4 * nn; i += blockDim.x) {
                    const int row = i / nn, col = i - row * nn;
                    const TabEntry e = sg.tab[(swar_ds(row) + sg.dsmax) * nn + col];
                    st4[i] = e.always ? 0xFFFFFFFFu : e.thr - 1u;
                }
            } else {
                for (int i = threadIdx.x; i < sg.tab_n; i += blockDim.x) stab[i] = sg.tab[i];
            }
            loaded = (int)w.x;
            __syncthreads();
        }
        // register copies: no aliasing with shared-memory stores
        const View3 v = view3(sg);
        Ctrl *const ctrl = sg.ctrl;
        const uint32_t key0 = sg.key0, key1 = sg.key1;
        const unsigned long long sweep = ctrl->sweep;
        const bool ref = v.ref != nullptr;
        Acc3 acc;
        if constexpr (kSwar) {   // 3D spin-1/2, 3D spin-1, 2D spin-1
            const int which = v.two_S == 1 ? 0 : (v.dims == 3 ? 1 : 2);
            if (which == 0) {
                if (ref) batch_w3_item<2, 1, 3, kColour, true, true>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
                else batch_w3_item<2, 1, 3, kColour, false, true>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
            } else if (which == 1) {
                if (ref) batch_w3_item<1, 2, 3, kColour, true, true>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
                else batch_w3_item<1, 2, 3, kColour, false, true>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
            } else {
                if (ref) batch_w3_item<1, 2, 2, kColour, true, true>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
                else batch_w3_item<1, 2, 2, kColour, false, true>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
            }
        } else {                 // per site: 3D spin-1/2 (4 sites per call), any other spin
            if (v.two_S == 1) {
                if (ref) batch_w3_item<2, 1, 3, kColour, true, false>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
                else batch_w3_item<2, 1, 3, kColour, false, false>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
            } else {
                if (ref) batch_w3_item<1, 0, 0, kColour, true, false>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
                else batch_w3_item<1, 0, 0, kColour, false, false>(v, key0, key1, sweep, stab, st4, w.y, passes, acc);
            }
        }
        if constexpr (kColour == 1) {
            unsigned long long *slot = series_slot(ctrl, sweep);
            long long t;
            t = block_sum_ll((long long)acc.bond, red);
            if (threadIdx.x == 0) add_counter(slot + 0, t);
            t = block_sum_ll((long long)acc.mag, red);
            if (threadIdx.x == 0) add_counter(slot + 1, t);
            t = block_sum_ll((long long)acc.up, red);
            if (threadIdx.x == 0) add_counter(slot + 2, t);
            if (ref) {
                t = block_sum_ll((long long)acc.acf, red);
                if (threadIdx.x == 0) add_counter(acf_slot(ctrl, sweep), t);
            }
        }
        __syncthreads();
    }
    dep_launch();   // no items left: the next kernel may be scheduled
}

}  // namespace

bool wide3_swar(const Geom &g)
{
    return g.tab_strict && (g.two_S == 1 || g.two_S == 2) && (g.dims == 3 || g.two_S == 2);
}

// Rows per thread for the 3D / spin-S (or Potts) items of a batch phase
// whose lattices of that kind hold chunk_rows (row, chunk column) pairs in
// all: 4 to 32 rows, as many as leave at least 4 items per CTA of one wave
// (2 CTAs on 152 SMs).  Long items pay their set-up (Philox keys, counter
// reduction) once per many chunks and keep two chunks in flight for
// longer; enough items keep the SMs level.  (16 lattices of 256^3: 32
// rows, 476 upd/ns, against 432 at 8 rows and 464 at 16; 16 Potts
// lattices of 1024^2: 4 rows, 264 upd/ns, against 226 at 2 and 257 at 8.)
int batch_item_passes(uint64_t chunk_rows)
{
    const uint64_t per = chunk_rows / ((uint64_t)kThreads * 4u * 2u * 152u);
    int p = 4;
    while (p < 32 && (uint64_t)(2 * p) <= per) p *= 2;
    return p;
}

int wide3_items(const Geom &g, int passes)
{
    const ColItemShape sh = col_item_shape(g.half, g.rows, (uint32_t)passes);
    return (int)(((g.rows + sh.br - 1u) / sh.br) * sh.nseg);
}

int batch_wide3_grid(bool swar)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (swar) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_wide3<1, true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_wide3<1, false>, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_wide3(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int colour, bool swar, int passes, int grid, cudaStream_t st)
{
    using K = void (*)(const Geom *, const uint2 *, int, unsigned *, uint32_t);
    static const K kern[2][2] = {{k_batch_wide3<0, false>, k_batch_wide3<1, false>},
                                 {k_batch_wide3<0, true>, k_batch_wide3<1, true>}};
    return launch_pdl(kern[swar ? 1 : 0][colour ? 1 : 0], (unsigned)grid, kThreads, st, geoms, items, n_items,
                      next_item, (uint32_t)passes);
}

bool wide3_supported(const Geom &g)
{
    return g.model == LAT_ISING && (g.dims == 3 || g.two_S >= 2) && (g.L % 16) == 0 &&
           g.bits[0] == nullptr && g.cpl == nullptr && g.tab_n <= kMaxTab;
}

cudaError_t launch_sweep_wide3(const Geom &g, int off, cudaStream_t st)
{
    // instantiations: 3D spin-1/2, 3D spin-1, 2D spin-1 (each byte-parallel
    // when the table has no never-accept entry, else per site), any other
    // spin-S; each colour, with and without a reference state
    const int base = g.two_S == 1 ? 0 : (g.two_S == 2 ? (g.dims == 3 ? 1 : 2) : 3);
    const int which = base < 3 && g.tab_strict ? base + 4 : base;
    const int ref = g.ref != nullptr ? 1 : 0;
    using K = void (*)(Geom, int);
    static const K kern[7][2][2] = {
        {{k_wide3_pipe<2, 1, 3, 0, false>, k_wide3_pipe<2, 1, 3, 1, false>},
         {k_wide3_pipe<2, 1, 3, 0, true>, k_wide3_pipe<2, 1, 3, 1, true>}},
        {{k_wide3_pipe<1, 2, 3, 0, false>, k_wide3_pipe<1, 2, 3, 1, false>},
         {k_wide3_pipe<1, 2, 3, 0, true>, k_wide3_pipe<1, 2, 3, 1, true>}},
        {{k_wide3_pipe<1, 2, 2, 0, false>, k_wide3_pipe<1, 2, 2, 1, false>},
         {k_wide3_pipe<1, 2, 2, 0, true>, k_wide3_pipe<1, 2, 2, 1, true>}},
        {{k_wide3_pipe<1, 0, 0, 0, false>, k_wide3_pipe<1, 0, 0, 1, false>},
         {k_wide3_pipe<1, 0, 0, 0, true>, k_wide3_pipe<1, 0, 0, 1, true>}},
        {{k_wide3_pipe<2, 1, 3, 0, false, true>, k_wide3_pipe<2, 1, 3, 1, false, true>},
         {k_wide3_pipe<2, 1, 3, 0, true, true>, k_wide3_pipe<2, 1, 3, 1, true, true>}},
        {{k_wide3_pipe<1, 2, 3, 0, false, true>, k_wide3_pipe<1, 2, 3, 1, false, true>},
         {k_wide3_pipe<1, 2, 3, 0, true, true>, k_wide3_pipe<1, 2, 3, 1, true, true>}},
        {{k_wide3_pipe<1, 2, 2, 0, false, true>, k_wide3_pipe<1, 2, 2, 1, false, true>},
         {k_wide3_pipe<1, 2, 2, 0, true, true>, k_wide3_pipe<1, 2, 2, 1, true, true>}}};
    static int resident[7] = {0, 0, 0, 0, 0, 0, 0};
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
        cudaError_t e = launch_pdl(kern[which][ref][colour], blocks, kThreads, st, g, off);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lat
