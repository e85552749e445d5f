// kernels_potts.cu -- two launches per sweep (one per colour, the kernel
// boundary being the device-wide barrier of §III.A steps 6-7) for the
// q-state Potts model (the remark closing §III.A: the method carries over to it),
// int8 labels 0..q-1 in the checkerboard-planar layout, 2D or 3D, L a
// multiple of 16.
//
// A thread owns 8 consecutive same-colour sites of one plane row (one
// 8-byte load per row).  The equal-neighbour counts of the old and of the
// proposed labels come from byte-wise equality masks of whole neighbour
// words, and the table index (df + 1) * nn + (dn + nmax) is formed for the
// 8 sites at once with byte-wise adds (every byte stays below 64, so no
// carry crosses a byte).  Per site remain the proposal, one table lookup
// and the acceptance compare.  Draws come from the same Philox groups as
// the generic kernel (4 sites per call for q = 2, 2 for q >= 3).  The
// kernels (solo and batched) read s[sweep & 1] and write s[(sweep+1) & 1]
// without copying a plane (colour 1 takes the new colour-0 labels from the
// new buffer).  Colour 1 reduces the sweep's counters (equal-neighbour
// bonds, sites in state 0, the others, and the overlap with a reference
// state).
#include <algorithm>

#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxTab = 39;   // 3 * (2 * nmax + 1) with nmax = 6 (3D)

// 0x01 in every byte where a and b hold the same label, else 0x00 (labels
// below 128: the XOR of two bytes plus 0x7F sets bit 7 exactly when they
// differ, without a carry into the next byte).
LAT_D uint32_t eq_bytes(uint32_t a, uint32_t b)
{
    return (~((a ^ b) + 0x7F7F7F7Fu) >> 7) & 0x01010101u;
}

LAT_D int byte_sum(uint32_t x)
{
    const uint32_t s = (x & 0x00FF00FFu) + ((x >> 8) & 0x00FF00FFu);
    return (int)((s & 0xFFFFu) + (s >> 16));
}

// 0xFF in byte i for bit i of a 4-bit mask.
LAT_D uint32_t spread4(uint32_t m) { return ((m * 0x00204081u) & 0x01010101u) * 0xFFu; }

struct AccP {
    int bond = 0, zero = 0, other = 0, acf = 0;
};

// The fields of a Geom that this kernel reads, small enough for registers.
struct ViewP {
    int L, two_S, nn, nmax;
    uint32_t G, half;
    uint64_t plane;
    int8_t *s0, *s1;
    const int8_t *ref;
};

LAT_D ViewP viewp(const Geom &g)
{
    ViewP v;
    v.L = g.L;
    v.two_S = g.two_S;
    v.nn = g.nn;
    v.nmax = g.nmax;
    v.G = g.G;
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
// flight -- the next chunk's loads and Philox draws in the same block as
// this chunk's step.  Colour 0 reads both planes of the old buffer and
// writes plane 0 of the new one; colour 1 reads its own old labels from the
// old buffer and the new colour-0 labels from the new one and writes plane
// 1: no plane is copied.  Same chunks and draws as the generic kernel.
// ---------------------------------------------------------------------
template <int D>
struct PIn {
    uint2 S, O;
    uint2 Nb[2 * D];   // entries 2.. : north, south (and z-1, z+1); 0, 1 filled by the step
    uint32_t nb;       // the other plane's word west (x = 2j) or east (x = 2j+1) of the chunk
};

template <int D, int kColour>
LAT_D void potts_load(const int8_t *pS, const int8_t *pO, uint32_t half, uint32_t L, uint32_t r, uint32_t y,
                      uint32_t z, uint32_t k, uint32_t wprev, uint32_t wnext, PIn<D> &in)
{
    auto ld = [&](const int8_t *p, uint32_t rr) { return *reinterpret_cast<const uint2 *>(p + (size_t)rr * half + 8 * k); };
    in.S = ld(pS, r);
    in.O = ld(pO, r);
    in.Nb[2] = ld(pO, (y == 0 ? L - 1 : y - 1) + L * z);
    in.Nb[3] = ld(pO, (y == L - 1 ? 0 : y + 1) + L * z);
    if constexpr (D == 3) {
        in.Nb[4] = ld(pO, y + L * (z == 0 ? L - 1 : z - 1));
        in.Nb[5] = ld(pO, y + L * (z == L - 1 ? 0 : z + 1));
    }
    const bool p1 = ((kColour + y + z) & 1) != 0;
    in.nb = reinterpret_cast<const uint32_t *>(pO + (size_t)r * half)[p1 ? wnext : wprev];
}

template <int SH, int D, int kColour, bool kRef>
LAT_D void potts_step(const ViewP &g, const TabEntry *stab, int8_t *dS, const int8_t *r1, const int8_t *r0,
                      uint32_t r, uint32_t y, uint32_t z, uint32_t k, PIn<D> &in, const U4 (&u)[8 >> SH], AccP &acc)
{
    const uint32_t half = g.half;
    const uint2 S = in.S, O = in.O;
    if (((kColour + y + z) & 1) == 0) {   // west is j-1 of the other plane, east is j
        in.Nb[0] = make_uint2(__funnelshift_l(in.nb, O.x, 8), __funnelshift_l(O.x, O.y, 8));
        in.Nb[1] = O;
    } else {                              // west is j, east is j+1
        in.Nb[0] = O;
        in.Nb[1] = make_uint2(__funnelshift_r(O.x, O.y, 8), __funnelshift_r(O.y, in.nb, 8));
    }
    uint2 Sn = make_uint2(0u, 0u);
    if constexpr (SH == 2) {
        Sn = make_uint2(S.x ^ 0x01010101u, S.y ^ 0x01010101u);
    } else {
        const uint32_t q1 = (uint32_t)g.two_S;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t sw = q < 4 ? S.x : S.y;
            const int sh8 = 8 * (q & 3);
            const uint32_t k_old = (sw >> sh8) & 0xFFu;
            const uint32_t u_prop = word_of(u[q >> 1], 2 * (q & 1) + 1);
            uint32_t k_new = k_old + 1u + (uint32_t)(((uint64_t)u_prop * (uint64_t)q1) >> 32);
            if (k_new > q1) k_new -= q1 + 1u;
            if (q < 4) Sn.x |= k_new << sh8;
            else Sn.y |= k_new << sh8;
        }
    }
    const uint32_t ones = 0x01010101u;
    uint32_t c_old_lo = 0, c_old_hi = 0, c_new_lo = 0, c_new_hi = 0;
#pragma unroll
    for (int d = 0; d < 2 * D; ++d) {
        c_old_lo += eq_bytes(in.Nb[d].x, S.x);
        c_old_hi += eq_bytes(in.Nb[d].y, S.y);
        c_new_lo += eq_bytes(in.Nb[d].x, Sn.x);
        c_new_hi += eq_bytes(in.Nb[d].y, Sn.y);
    }
    const uint32_t nn = (uint32_t)g.nn, nmax = (uint32_t)g.nmax;
    const uint32_t idx_lo = (eq_bytes(Sn.x, 0u) + ones - eq_bytes(S.x, 0u)) * nn + (c_new_lo + nmax * ones - c_old_lo);
    const uint32_t idx_hi = (eq_bytes(Sn.y, 0u) + ones - eq_bytes(S.y, 0u)) * nn + (c_new_hi + nmax * ones - c_old_hi);
    uint32_t am = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t iw = q < 4 ? idx_lo : idx_hi;
        const TabEntry e = stab[(iw >> (8 * (q & 3))) & 0xFFu];
        const uint32_t u_acc = SH == 2 ? word_of(u[q >> 2], q & 3) : word_of(u[q >> 1], 2 * (q & 1));
        if (e.always || u_acc < e.thr) am |= 1u << q;
    }
    const uint32_t m_lo = spread4(am & 0xFu), m_hi = spread4(am >> 4);
    const uint2 Sf = make_uint2(S.x ^ ((S.x ^ Sn.x) & m_lo), S.y ^ ((S.y ^ Sn.y) & m_hi));
    *reinterpret_cast<uint2 *>(dS + (size_t)r * half + 8 * k) = Sf;
    if constexpr (kColour == 1) {
        uint32_t eq = 0;
#pragma unroll
        for (int d = 0; d < 2 * D; ++d) eq += eq_bytes(in.Nb[d].x, Sf.x) + eq_bytes(in.Nb[d].y, Sf.y);
        acc.bond += byte_sum(eq);
        const int z0 = byte_sum(eq_bytes(Sf.x, 0u) + eq_bytes(Sf.y, 0u) + eq_bytes(O.x, 0u) + eq_bytes(O.y, 0u));
        acc.zero += z0;
        acc.other += 16 - z0;
        if constexpr (kRef) {
            const uint2 R1 = *reinterpret_cast<const uint2 *>(r1 + (size_t)r * half + 8 * k);
            const uint2 R0 = *reinterpret_cast<const uint2 *>(r0 + (size_t)r * half + 8 * k);
            acc.acf += byte_sum(eq_bytes(Sf.x, R1.x) + eq_bytes(Sf.y, R1.y) + eq_bytes(O.x, R0.x) +
                                eq_bytes(O.y, R0.y));
        }
    }
}

template <int SH, int D, int kColour, bool kRef>
__global__ void __launch_bounds__(kThreads, 2) k_potts_pipe(Geom g, int off)
{
    __shared__ TabEntry stab[kMaxTab];
    __shared__ long long red[kThreads / 32];
    if (threadIdx.x < (unsigned)g.tab_n) stab[threadIdx.x] = g.tab[threadIdx.x];
    __syncthreads();
    dep_wait();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const ViewP v = viewp(g);
    const int8_t *old = (sweep & 1) ? v.s1 : v.s0;
    int8_t *nw = (sweep & 1) ? v.s0 : v.s1;
    const uint32_t plane = (uint32_t)v.plane;
    const int8_t *pS = old + (size_t)kColour * plane;
    const int8_t *pO = (kColour == 0 ? old : nw) + (size_t)(1 - kColour) * plane;
    int8_t *dS = nw + (size_t)kColour * plane;
    const int8_t *r1 = v.ref ? v.ref + plane : nullptr, *r0 = v.ref;
    AccP acc;
    const uint32_t cpr = v.half >> 3;   // 8-site chunks per plane row
    const uint32_t rows = g.rows, L = (uint32_t)v.L;
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
        PIn<D> A, B;
        U4 uA[kCalls], uB[kCalls];
        potts_load<D, kColour>(pS, pO, v.half, L, r, y, z, k, wprev, wnext, A);
        draws(r, uA);
        for (;;) {
            const uint32_t r1_ = r + rs;
            uint32_t y1 = y, z1 = z;
            step_row(y1, z1);
            if (r1_ >= rows) {
                potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, r, y, z, k, A, uA, acc);
                break;
            }
            potts_load<D, kColour>(pS, pO, v.half, L, r1_, y1, z1, k, wprev, wnext, B);
            draws(r1_, uB);
            potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, r, y, z, k, A, uA, acc);
            const uint32_t r2 = r1_ + rs;
            uint32_t y2 = y1, z2 = z1;
            step_row(y2, z2);
            if (r2 >= rows) {
                potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, r1_, y1, z1, k, B, uB, acc);
                break;
            }
            potts_load<D, kColour>(pS, pO, v.half, L, r2, y2, z2, k, wprev, wnext, A);
            draws(r2, uA);
            potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, r1_, y1, z1, k, B, uB, acc);
            r = r2;
            y = y2;
            z = z2;
        }
    }
    dep_launch();   // main work done: the next kernel may be scheduled
    if constexpr (kColour == 1) {
        unsigned long long *slot = series_slot(g.ctrl, sweep);
        long long s;
        s = block_sum_ll((long long)acc.bond, red);
        if (threadIdx.x == 0) add_counter(slot + 0, s);
        s = block_sum_ll((long long)acc.zero, red);
        if (threadIdx.x == 0) add_counter(slot + 1, s);
        s = block_sum_ll((long long)acc.other, red);
        if (threadIdx.x == 0) add_counter(slot + 2, s);
        if constexpr (kRef) {
            s = block_sum_ll((long long)acc.acf, red);
            if (threadIdx.x == 0) add_counter(acf_slot(g.ctrl, sweep), s);
        }
    }
}

// Batched form: a persistent grid takes (lattice, item) pairs from an
// atomic counter; an item is a band of plane rows x a segment of chunk
// columns of one colour of one lattice (col_item_shape), each thread walking
// its column down the band with two chunks in flight and the same no-copy
// convention as the solo kernel.  The descriptor and table are reloaded only
// when a CTA moves to another lattice (items are ordered by lattice).
template <int SH, int D, int kColour, bool kRef>
LAT_D void batch_potts_item(const ViewP &v, uint32_t rows, uint32_t key0, uint32_t key1, unsigned long long sweep,
                            const TabEntry *stab, uint32_t item, uint32_t passes, AccP &acc)
{
    const ColItemShape sh = col_item_shape(v.half, rows, passes);
    const uint32_t L = (uint32_t)v.L;
    const uint32_t band = item / sh.nseg, seg = item - band * sh.nseg;
    const uint32_t r_end = min(rows, band * sh.br + sh.br);
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
    const uint32_t wprev = wrap_once(2 * k - 1 + nwr, nwr), wnext = wrap_once(2 * k + 2, nwr);
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
    PIn<D> A, B;
    U4 uA[kCalls], uB[kCalls];
    potts_load<D, kColour>(pS, pO, v.half, L, r, y, z, k, wprev, wnext, A);
    draws(r, uA);
    for (;;) {
        const uint32_t ra = r + sh.rsb;
        uint32_t ya = y, za = z;
        step_row(ya, za);
        if (ra >= r_end) {
            potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, r, y, z, k, A, uA, acc);
            break;
        }
        potts_load<D, kColour>(pS, pO, v.half, L, ra, ya, za, k, wprev, wnext, B);
        draws(ra, uB);
        potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, r, y, z, k, A, uA, acc);
        const uint32_t rb = ra + sh.rsb;
        uint32_t yb = ya, zb = za;
        step_row(yb, zb);
        if (rb >= r_end) {
            potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, ra, ya, za, k, B, uB, acc);
            break;
        }
        potts_load<D, kColour>(pS, pO, v.half, L, rb, yb, zb, k, wprev, wnext, A);
        draws(rb, uA);
        potts_step<SH, D, kColour, kRef>(v, stab, dS, r1, r0, ra, ya, za, k, B, uB, acc);
        r = rb;
        y = yb;
        z = zb;
    }
}

template <int kColour>
__global__ void __launch_bounds__(kThreads, 2) k_batch_potts(const Geom *geoms, const uint2 *items, int n_items,
                                                            unsigned *next_item, uint32_t passes)
{
    __shared__ TabEntry stab[kMaxTab];
    __shared__ long long red[kThreads / 32];
    __shared__ Geom sg;
    __shared__ int cur;
    int loaded = -1;
    dep_wait();   // the work counter, sweep numbers and labels of the step before
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
            if (threadIdx.x < (unsigned)sg.tab_n) stab[threadIdx.x] = sg.tab[threadIdx.x];
            loaded = (int)w.x;
            __syncthreads();
        }
        // register copies: no aliasing with shared-memory stores
        const ViewP v = viewp(sg);
        Ctrl *const ctrl = sg.ctrl;
        const uint32_t rows = sg.rows, key0 = sg.key0, key1 = sg.key1;
        const int which = (sg.two_S == 1 ? 0 : 2) + (sg.dims == 3 ? 1 : 0);
        const unsigned long long sweep = ctrl->sweep;
        const bool ref = v.ref != nullptr;
        AccP acc;
        switch (which) {
        case 0:
            if (ref) batch_potts_item<2, 2, kColour, true>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            else batch_potts_item<2, 2, kColour, false>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            break;
        case 1:
            if (ref) batch_potts_item<2, 3, kColour, true>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            else batch_potts_item<2, 3, kColour, false>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            break;
        case 2:
            if (ref) batch_potts_item<1, 2, kColour, true>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            else batch_potts_item<1, 2, kColour, false>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            break;
        default:
            if (ref) batch_potts_item<1, 3, kColour, true>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
            else batch_potts_item<1, 3, kColour, false>(v, rows, key0, key1, sweep, stab, w.y, passes, acc);
        }
        if constexpr (kColour == 1) {
            unsigned long long *slot = series_slot(ctrl, sweep);
            long long s;
            s = block_sum_ll((long long)acc.bond, red);
            if (threadIdx.x == 0) add_counter(slot + 0, s);
            s = block_sum_ll((long long)acc.zero, red);
            if (threadIdx.x == 0) add_counter(slot + 1, s);
            s = block_sum_ll((long long)acc.other, red);
            if (threadIdx.x == 0) add_counter(slot + 2, s);
            if (ref) {
                s = block_sum_ll((long long)acc.acf, red);
                if (threadIdx.x == 0) add_counter(acf_slot(ctrl, sweep), s);
            }
        }
        __syncthreads();
    }
    dep_launch();   // no items left: the next kernel may be scheduled
}

}  // namespace

int potts_items(const Geom &g, int passes)
{
    const ColItemShape sh = col_item_shape(g.half, g.rows, (uint32_t)passes);
    return (int)(((g.rows + sh.br - 1u) / sh.br) * sh.nseg);
}

int batch_potts_grid()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_potts<1>, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_batch_potts(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int colour, int passes, int grid, cudaStream_t st)
{
    using K = void (*)(const Geom *, const uint2 *, int, unsigned *, uint32_t);
    const K kern = colour ? k_batch_potts<1> : k_batch_potts<0>;
    return launch_pdl(kern, (unsigned)grid, kThreads, st, geoms, items, n_items, next_item, (uint32_t)passes);
}

bool potts_supported(const Geom &g)
{
    return g.model == LAT_POTTS && (g.L % 16) == 0 && g.bits[0] == nullptr && g.cpl == nullptr &&
           g.tab_n <= kMaxTab && g.two_S <= 8;
}

cudaError_t launch_sweep_potts(const Geom &g, int off, cudaStream_t st)
{
    // instantiations: q = 2 and q >= 3, each in 2D and 3D; each colour,
    // with and without a reference state
    const int which = (g.two_S == 1 ? 0 : 2) + (g.dims == 3 ? 1 : 0);
    const int ref = g.ref != nullptr ? 1 : 0;
    using K = void (*)(Geom, int);
    static const K kern[4][2][2] = {
        {{k_potts_pipe<2, 2, 0, false>, k_potts_pipe<2, 2, 1, false>},
         {k_potts_pipe<2, 2, 0, true>, k_potts_pipe<2, 2, 1, true>}},
        {{k_potts_pipe<2, 3, 0, false>, k_potts_pipe<2, 3, 1, false>},
         {k_potts_pipe<2, 3, 0, true>, k_potts_pipe<2, 3, 1, true>}},
        {{k_potts_pipe<1, 2, 0, false>, k_potts_pipe<1, 2, 1, false>},
         {k_potts_pipe<1, 2, 0, true>, k_potts_pipe<1, 2, 1, true>}},
        {{k_potts_pipe<1, 3, 0, false>, k_potts_pipe<1, 3, 1, false>},
         {k_potts_pipe<1, 3, 0, true>, k_potts_pipe<1, 3, 1, true>}}};
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
        cudaError_t e = launch_pdl(kern[which][ref][colour], blocks, kThreads, st, g, off);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lat
