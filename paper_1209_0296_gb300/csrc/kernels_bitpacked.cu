// kernels_bitpacked.cu -- the bit-packed spin-1/2 layout: conversion to and
// from int8 spins, and (below) its sweep kernel.
//
// Layout: for colour c and row y, bit (j & 31) of word (j >> 5) holds the
// j-th colour-c site of the row (x = 2j + ((c + y) & 1)), i.e. entry j of
// row y of colour plane c of the planar int8 layout; a set bit is an up
// spin (+1).  Words per row bw = ceil((L/2) / 32).
#include <algorithm>

#include "lattice_internal.cuh"

namespace lat {

namespace {

constexpr int kThreads = 256;

// planar int8 -> bits: word k of plane c row y holds sites j = 32k .. 32k+31.
__global__ void k_pack(Geom g, const int8_t *planar, uint32_t *bits)
{
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t total = 2ull * g.L * g.bw;
    if (t >= total) return;
    const uint32_t k = (uint32_t)(t % g.bw);
    const uint64_t row = t / g.bw;  // c * L + y
    const int8_t *src = planar + row * g.half;
    uint32_t w = 0;
    for (uint32_t b = 0; b < 32; ++b) {
        const uint32_t j = 32 * k + b;
        if (j >= g.half) break;
        if (src[j] > 0) w |= 1u << b;
    }
    bits[t] = w;
}

__global__ void k_unpack(Geom g, const uint32_t *bits, int8_t *planar)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    const uint64_t row = i / g.half;  // c * L + y
    const uint32_t j = (uint32_t)(i % g.half);
    const uint32_t w = bits[row * g.bw + (j >> 5)];
    planar[i] = ((w >> (j & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
}


// Bits 4q..4q+3 of x spread to bit 0 of bytes 0..3.
LAT_D uint32_t spread_nibble(uint32_t x, int q) { return (((x >> (4 * q)) & 0xFu) * 0x00204081u) & 0x01010101u; }

// One colour of one sweep on the bit-packed planes (L % 64 == 0): a word =
// 32 same-colour sites of one plane row = 8 Philox groups; neighbour
// counts of all 32 sites at once, bit-sliced.  Persistent,
// software-pipelined: one wave of CTAs; each thread walks
// one word column k down the rows y0, y0 + rs, ... with the next row's five
// loads in flight while it updates this row's word (the eight Philox calls
// of a word need no loads and interleave with its Metropolis step).
// Colour 0 reads both planes of the old buffer and writes plane 0 of the
// new one; colour 1 reads its own old word from the old buffer and the new
// colour-0 words from the new one, and writes plane 1: no plane is copied.
struct BitsIn {
    uint32_t S, O, U, D, nb;   // nb: the other plane's word west (x = 2j) or east (x = 2j+1) of O
};

template <bool kNE, int kColour>
__global__ void __launch_bounds__(kThreads, 3) k_bits_pipe(Geom g, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ long long red[kThreads / 32];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    dep_wait();
    constexpr int oc = 1 - kColour;
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const uint32_t *old = g.bits[sweep & 1];
    uint32_t *nw = g.bits[(sweep + 1) & 1];
    const uint32_t L = (uint32_t)g.L, bw = g.bw;
    const uint32_t *pS = old + (size_t)kColour * L * bw;
    const uint32_t *pO = (kColour == 0 ? old : nw) + (size_t)oc * L * bw;
    uint32_t *dS = nw + (size_t)kColour * L * bw;
    const uint32_t rs = (gridDim.x * blockDim.x) / bw;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t y = gt / bw;
    const uint32_t k = gt - y * bw;
    long long bond = 0, mag = 0, up = 0, unfl = 0, acf = 0;
    if (y < rs && y < L) {
        const uint32_t km = k == 0 ? bw - 1 : k - 1, kp = k == bw - 1 ? 0 : k + 1;
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        const char *tb = reinterpret_cast<const char *>(sthr);
        auto load = [&](uint32_t yy, BitsIn &in) {
            const uint32_t ym = yy == 0 ? L - 1 : yy - 1, yp = yy == L - 1 ? 0 : yy + 1;
            in.S = pS[(size_t)yy * bw + k];
            in.O = pO[(size_t)yy * bw + k];
            in.U = pO[(size_t)ym * bw + k];
            in.D = pO[(size_t)yp * bw + k];
            in.nb = pO[(size_t)yy * bw + (((kColour + yy) & 1) ? kp : km)];
        };
        auto step = [&](uint32_t yy, const BitsIn &in) {
            uint32_t Lf, R;
            if (((kColour + yy) & 1) == 0) {   // x = 2j: west is j-1, east is j
                Lf = (in.O << 1) | (in.nb >> 31);
                R = in.O;
            } else {                           // x = 2j+1: west is j, east is j+1
                Lf = in.O;
                R = (in.O >> 1) | (in.nb << 31);
            }
            const uint32_t Ud = ~in.U, Dd = ~in.D, Ld = ~Lf, Rd = ~R, Sd = ~in.S;
            const uint32_t s1 = Ud ^ Dd ^ Ld;
            const uint32_t c1 = (Ud & Dd) | (Ud & Ld) | (Dd & Ld);
            const uint32_t b0 = s1 ^ Rd;
            const uint32_t b1 = c1 ^ (s1 & Rd);
            const uint32_t b2 = c1 & s1 & Rd;
            const uint32_t lock = kNE ? (Ud | Rd) : 0u;   // §III.B: north and east must be up
            uint32_t flip = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t idx = (spread_nibble(b0, q) << 2) | (spread_nibble(b1, q) << 3) |
                                     (spread_nibble(b2, q) << 4) | (spread_nibble(Sd, q) << 5);
                uint32_t t0 = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
                uint32_t t1 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
                uint32_t t2 = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
                uint32_t t3 = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
                uint32_t lk = 0;
                if (kNE) {
                    lk = (lock >> (4 * q)) & 0xFu;
                    t0 |= 0u - (lk & 1u);
                    t1 |= 0u - ((lk >> 1) & 1u);
                    t2 |= 0u - ((lk >> 2) & 1u);
                    t3 |= 0u - ((lk >> 3) & 1u);
                }
                uint32_t acc = 0xFu;
                if (!kNE || (t0 & t1 & t2 & t3) != 0xFFFFFFFFu) {
                    const uint32_t grp = yy * g.G + 8u * k + (uint32_t)q;
                    const U4 u = philox_item(pp, grp, (uint32_t)kColour);
                    acc = (u.x <= t0 ? 1u : 0u) | (u.y <= t1 ? 2u : 0u) | (u.z <= t2 ? 4u : 0u) |
                          (u.w <= t3 ? 8u : 0u);
                }
                if (kNE) acc &= ~lk;
                flip |= acc << (4 * q);
            }
            const uint32_t Sn = in.S ^ flip;
            dS[(size_t)yy * bw + k] = Sn;
            uint32_t fl_c_pop = 0, fl_o_pop = 0;
            if (kNE) {
                uint2 *fp = reinterpret_cast<uint2 *>(g.flags + ((size_t)kColour * L + yy) * g.G + 8u * k);
                uint2 f = *fp;
                uint32_t lo = 0, hi = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) lo |= ((flip >> (4 * q)) & 0xFu) << (8 * q);
#pragma unroll
                for (int q = 0; q < 4; ++q) hi |= ((flip >> (16 + 4 * q)) & 0xFu) << (8 * q);
                f.x |= lo;
                f.y |= hi;
                *fp = f;
                fl_c_pop = __popc(f.x) + __popc(f.y);
                if (kColour == 1) {
                    const uint2 fo =
                        *reinterpret_cast<const uint2 *>(g.flags + ((size_t)oc * L + yy) * g.G + 8u * k);
                    fl_o_pop = __popc(fo.x) + __popc(fo.y);
                }
            }
            if (kColour == 1) {
                const uint32_t Snd = ~Sn;
                const int uneq = __popc(Snd ^ Ud) + __popc(Snd ^ Dd) + __popc(Snd ^ Ld) + __popc(Snd ^ Rd);
                bond += 128 - 2 * uneq;
                const int downs = __popc(Snd) + __popc(~in.O);
                mag += 64 - 2 * downs;
                up += 64 - downs;
                unfl += 64 - (int)fl_c_pop - (int)fl_o_pop;
                if (g.ref_bits != nullptr) {
                    const uint32_t r1 = g.ref_bits[((size_t)1 * L + yy) * bw + k];
                    const uint32_t r0 = g.ref_bits[(size_t)yy * bw + k];
                    acf += 64 - 2 * (__popc(Sn ^ r1) + __popc(in.O ^ r0));
                }
            }
        };
        BitsIn A, B;
        load(y, A);
        for (;;) {
            const uint32_t y1 = y + rs;
            if (y1 >= L) {
                step(y, A);
                break;
            }
            load(y1, B);
            step(y, A);
            const uint32_t y2 = y1 + rs;
            if (y2 >= L) {
                step(y1, B);
                break;
            }
            load(y2, A);
            step(y1, B);
            y = y2;
        }
    }
    dep_launch();   // main work done: the next kernel may be scheduled
    if (kColour == 1) {
        unsigned long long *slot = series_slot(g.ctrl, sweep);
        long long v;
        v = block_sum_ll(bond, red);
        if (threadIdx.x == 0) add_counter(slot + 0, v);
        v = block_sum_ll(mag, red);
        if (threadIdx.x == 0) add_counter(slot + 1, v);
        v = block_sum_ll(up, red);
        if (threadIdx.x == 0) add_counter(slot + 2, v);
        if (kNE) {
            v = block_sum_ll(unfl, red);
            if (threadIdx.x == 0) add_counter(slot + 3, v);
        }
        if (g.ref_bits != nullptr) {
            v = block_sum_ll(acf, red);
            if (threadIdx.x == 0) add_counter(acf_slot(g.ctrl, sweep), v);
        }
    }
}

}  // namespace

cudaError_t launch_pack_bits(const Geom &g, const int8_t *planar, uint32_t *bits, cudaStream_t st)
{
    const uint64_t total = 2ull * g.L * g.bw;
    k_pack<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, planar, bits);
    return cudaGetLastError();
}

cudaError_t launch_unpack_bits(const Geom &g, const uint32_t *bits, int8_t *planar, cudaStream_t st)
{
    k_unpack<<<(unsigned)((g.N + kThreads - 1) / kThreads), kThreads, 0, st>>>(g, bits, planar);
    return cudaGetLastError();
}

cudaError_t launch_sweep_bitpacked(const Geom &g, int off, cudaStream_t st)
{
    const Geom k = tiled_geom(g);  // compact table in t' = thr - 1 form
    using K = void (*)(Geom, int);
    const bool ne = g.model == LAT_NE;
    const K c0 = ne ? k_bits_pipe<true, 0> : k_bits_pipe<false, 0>;
    const K c1 = ne ? k_bits_pipe<true, 1> : k_bits_pipe<false, 1>;
    // one wave: SMs x resident CTAs per SM (queried once per model)
    static int wave[2] = {0, 0};
    int &w = wave[ne ? 1 : 0];
    if (w == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, reinterpret_cast<const void *>(c1), kThreads, 0);
        w = sms * (per > 0 ? per : 1);
    }
    const uint64_t words = (uint64_t)g.L * g.bw;
    const unsigned blocks = (unsigned)std::min<uint64_t>((words + kThreads - 1) / kThreads, (uint64_t)w);
    cudaError_t e = launch_pdl(c0, blocks, kThreads, st, k, off);
    return e == cudaSuccess ? launch_pdl(c1, blocks, kThreads, st, k, off) : e;
}

bool bitpacked_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && (g.L % 64) == 0) || g.model == LAT_POTTS) return false;
    for (int k = 0; k < 16; ++k) {
        if ((k & 7) > 4) continue;
        if (!((g.always16 >> k) & 1u) && g.thr16[k] == 0u) return false;
    }
    return true;
}

}  // namespace lat
