// kernels_bitpacked.cu -- the bit-packed spin-1/2 layout: conversion to and
// from int8 spins, and (below) its sweep kernel.
//
// Layout: for colour c and row y, bit (j & 31) of word (j >> 5) holds the
// j-th colour-c site of the row (x = 2j + ((c + y) & 1)), i.e. entry j of
// row y of colour plane c of the planar int8 layout; a set bit is an up
// spin (+1).  Words per row bw = ceil((L/2) / 32).
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

// One colour of one sweep on the bit-packed planes (L % 64 == 0).  Thread =
// one 32-bit word of the colour-c plane of row y: 32 same-colour sites = 8
// Philox groups.  Colour 0 reads bits[sweep & 1] and writes the new colour-0
// word and a copy of the colour-1 word at the same index into
// bits[(sweep+1) & 1]; colour 1 then works in place there and accumulates
// the sweep's counters.
template <bool kNE>
__global__ void __launch_bounds__(kThreads, 4) k_bits_half(Geom g, int colour, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ long long red[kThreads / 32];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    const uint32_t *src = g.bits[sweep & 1];
    uint32_t *dst = g.bits[(sweep + 1) & 1];
    if (colour == 1) src = dst;
    const int L = g.L;
    const uint32_t bw = g.bw;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;   // L * bw < 2^26
    long long bond = 0, mag = 0, up = 0, unfl = 0, acf = 0;
    if (t < (uint32_t)L * bw) {
        const int y = (int)(t / bw);
        const int k = (int)(t - (uint32_t)y * bw);
        const int oc = 1 - colour;
        const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
        const int km = k == 0 ? (int)bw - 1 : k - 1, kp = k == (int)bw - 1 ? 0 : k + 1;
        auto W = [&](int c, int row, int col) { return src[((uint64_t)c * L + row) * bw + col]; };
        const uint32_t S = W(colour, y, k);   // set bit = up
        const uint32_t O = W(oc, y, k);
        const uint32_t U = W(oc, ym, k);      // north
        const uint32_t D = W(oc, yp, k);      // south
        uint32_t Lf, R;
        if (((colour + y) & 1) == 0) {        // x = 2j: west is j-1, east is j
            Lf = (O << 1) | (W(oc, y, km) >> 31);
            R = O;
        } else {                              // x = 2j+1: west is j, east is j+1
            Lf = O;
            R = (O >> 1) | (W(oc, y, kp) << 31);
        }
        // Down-neighbour counts of all 32 sites at once (bit-sliced).
        const uint32_t Ud = ~U, Dd = ~D, Ld = ~Lf, Rd = ~R, Sd = ~S;
        const uint32_t s1 = Ud ^ Dd ^ Ld;
        const uint32_t c1 = (Ud & Dd) | (Ud & Ld) | (Dd & Ld);
        const uint32_t b0 = s1 ^ Rd;
        const uint32_t b1 = c1 ^ (s1 & Rd);
        const uint32_t b2 = c1 & s1 & Rd;
        const uint32_t lock = kNE ? (Ud | Rd) : 0u;  // §III.B: north and east must be up
        PhiloxPre pp;
        philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
        const char *tb = reinterpret_cast<const char *>(sthr);
        uint32_t flip = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            // byte offsets (index sd<<3 | nd, 4 bytes per entry) of the 4 sites
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
            // Ising draws every group (a group that needs none is rare and
            // the branch costs more than it saves); a North-East group whose
            // sites are all locked or always-accepted skips its draw
            if (!kNE || (t0 & t1 & t2 & t3) != 0xFFFFFFFFu) {
                const uint32_t grp = (uint32_t)y * g.G + 8u * (uint32_t)k + (uint32_t)q;
                const U4 u = philox_item(pp, grp, (uint32_t)colour);
                acc = (u.x <= t0 ? 1u : 0u) | (u.y <= t1 ? 2u : 0u) | (u.z <= t2 ? 4u : 0u) |
                      (u.w <= t3 ? 8u : 0u);
            }
            if (kNE) acc &= ~lk;
            flip |= acc << (4 * q);
        }
        const uint32_t Sn = S ^ flip;
        dst[((uint64_t)colour * L + y) * bw + k] = Sn;
        if (colour == 0) dst[((uint64_t)1 * L + y) * bw + k] = O;
        uint32_t fl_c_pop = 0, fl_o_pop = 0;
        if (kNE) {
            // persistence bytes of the 8 groups of this word, bit q = site 4m+q
            uint2 *fp = reinterpret_cast<uint2 *>(g.flags + ((uint64_t)colour * L + y) * g.G + 8u * k);
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
            if (colour == 1) {
                const uint2 fo = *reinterpret_cast<const uint2 *>(
                    g.flags + ((uint64_t)oc * L + y) * g.G + 8u * k);
                fl_o_pop = __popc(fo.x) + __popc(fo.y);
            }
        }
        if (colour == 1) {
            const uint32_t Snd = ~Sn;
            const int uneq = __popc(Snd ^ Ud) + __popc(Snd ^ Dd) + __popc(Snd ^ Ld) + __popc(Snd ^ Rd);
            bond = 128 - 2 * uneq;
            const int downs = __popc(Snd) + __popc(~O);
            mag = 64 - 2 * downs;
            up = 64 - downs;
            unfl = 64 - (int)fl_c_pop - (int)fl_o_pop;
            if (g.ref_bits != nullptr) {   // overlap with the reference: 64 - 2 * (# differing)
                const uint32_t r1 = g.ref_bits[((uint64_t)1 * L + y) * bw + k];
                const uint32_t r0 = g.ref_bits[(uint64_t)y * bw + k];
                acf = 64 - 2 * (__popc(Sn ^ r1) + __popc(O ^ r0));
            }
        }
    }
    if (colour == 1) {
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
    const uint64_t words = (uint64_t)g.L * g.bw;
    const unsigned blocks = (unsigned)((words + kThreads - 1) / kThreads);
    for (int colour = 0; colour < 2; ++colour) {
        if (g.model == LAT_NE)
            k_bits_half<true><<<blocks, kThreads, 0, st>>>(k, colour, off);
        else
            k_bits_half<false><<<blocks, kThreads, 0, st>>>(k, colour, off);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
