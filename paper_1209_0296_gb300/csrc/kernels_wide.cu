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
    int bond = 0, mag = 0, up = 0, unfl = 0;
};

// Sweep colour `colour` of the 16-site chunk k of plane row y.
template <bool kNE>
LAT_D void wide_chunk(const SweepView g, const uint32_t *sthr, int colour, unsigned long long sweep,
                      const PhiloxPre &pp, int y, int k, Counts &cnt)
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
    const uint4 S4 = *reinterpret_cast<const uint4 *>(row(colour, y) + 16 * k);
    const uint4 O4 = *reinterpret_cast<const uint4 *>(row(oc, y) + 16 * k);
    const uint4 U4v = *reinterpret_cast<const uint4 *>(row(oc, ym) + 16 * k);   // north
    const uint4 D4v = *reinterpret_cast<const uint4 *>(row(oc, yp) + 16 * k);   // south
    const bool p1 = ((colour + y) & 1) != 0;
    uint32_t adj;
    {
        const uint32_t w = p1 ? (uint32_t)(4 * k + 4) : (uint32_t)(4 * k - 1 + nwr);
        adj = reinterpret_cast<const uint32_t *>(row(oc, y))[w % nwr];
    }
    const uint32_t S[4] = {S4.x, S4.y, S4.z, S4.w};
    const uint32_t O[4] = {O4.x, O4.y, O4.z, O4.w};
    const uint32_t U[4] = {U4v.x, U4v.y, U4v.z, U4v.w};
    const uint32_t D[4] = {D4v.x, D4v.y, D4v.z, D4v.w};
    uint32_t Lf[4], R[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (!p1) {  // x = 2j: west is j-1 of the other plane, east is j
            Lf[w] = __funnelshift_l(w == 0 ? adj : O[w - 1], O[w], 8);
            R[w] = O[w];
        } else {    // x = 2j+1: west is j, east is j+1
            Lf[w] = O[w];
            R[w] = __funnelshift_r(O[w], w == 3 ? adj : O[w + 1], 8);
        }
    }
    uint32_t t[4][4], locked[4];
    bool need = false;
    const char *tb = reinterpret_cast<const char *>(sthr);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t s1 = U[w] ^ D[w] ^ Lf[w];
        const uint32_t c1 = (U[w] & D[w]) | (U[w] & Lf[w]) | (D[w] & Lf[w]);
        const uint32_t b0 = s1 ^ R[w];
        const uint32_t b1 = c1 ^ (s1 & R[w]);
        const uint32_t b2 = c1 & s1 & R[w];
        // byte offset into the 16-entry table (index sd<<3 | nd, 4 bytes each)
        const uint32_t idx = (b0 & 0x04040404u) | (b1 & 0x08080808u) | (b2 & 0x10101010u) |
                             (S[w] & 0x20202020u);
        t[w][0] = *reinterpret_cast<const uint32_t *>(tb + (idx & 0xFFu));
        t[w][1] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 8) & 0xFFu));
        t[w][2] = *reinterpret_cast<const uint32_t *>(tb + ((idx >> 16) & 0xFFu));
        t[w][3] = *reinterpret_cast<const uint32_t *>(tb + (idx >> 24));
        locked[w] = 0;
        if (kNE) {
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
    U4 u[4] = {U4{0, 0, 0, 0}, U4{0, 0, 0, 0}, U4{0, 0, 0, 0}, U4{0, 0, 0, 0}};
    if (need) {
        const uint32_t g0 = (uint32_t)y * g.G + 4u * (uint32_t)k;
#pragma unroll
        for (int w = 0; w < 4; ++w) u[w] = philox_item(pp, g0 + (uint32_t)w, (uint32_t)colour);
    }
    uint32_t Sn[4], chg = 0;
    const uint32_t M1 = 0x02020202u;
    uint32_t ue = 0, dn = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t acc = (u[w].x <= t[w][0] ? 1u : 0u) | (u[w].y <= t[w][1] ? 2u : 0u) |
                             (u[w].z <= t[w][2] ? 4u : 0u) | (u[w].w <= t[w][3] ? 8u : 0u);
        uint32_t F = ((acc * 0x00204081u) & 0x01010101u) * 0xFEu;  // 0xFE at flipped sites
        if (kNE) {
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
    *reinterpret_cast<uint4 *>(dst + (uint64_t)colour * g.plane + (uint64_t)y * half + 16 * k) =
        make_uint4(Sn[0], Sn[1], Sn[2], Sn[3]);
    if (colour == 0)
        *reinterpret_cast<uint4 *>(dst + (uint64_t)g.plane + (uint64_t)y * half + 16 * k) = O4;
    int unfl = 0;
    if (kNE) {
        // persistence bytes of the 4 groups (bit q = site 4m+q)
        uint32_t *fp = reinterpret_cast<uint32_t *>(g.flags + ((uint64_t)colour * L + y) * g.G + 4u * k);
        const uint32_t f = *fp | chg;
        *fp = f;
        if (colour == 1) {
            const uint32_t fo =
                *reinterpret_cast<const uint32_t *>(g.flags + ((uint64_t)oc * L + y) * g.G + 4u * k);
            unfl = 32 - __popc(f) - __popc(fo);
        }
    }
    if (colour == 1) {
        const int d2 = byte_sum(dn);
        cnt.bond += 64 - byte_sum(ue);
        cnt.mag += 32 - d2;
        cnt.up += 32 - (d2 >> 1);
        cnt.unfl += unfl;
    }
}

LAT_D void flush(const SweepView &g, unsigned long long sweep, const Counts &c, bool ne, int (*red)[4])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rb = __reduce_add_sync(0xffffffffu, c.bond);
    const int rm = __reduce_add_sync(0xffffffffu, c.mag);
    const int ru = __reduce_add_sync(0xffffffffu, c.up);
    const int rf = __reduce_add_sync(0xffffffffu, c.unfl);
    if (lane == 0) {
        red[warp][0] = rb;
        red[warp][1] = rm;
        red[warp][2] = ru;
        red[warp][3] = rf;
    }
    __syncthreads();
    if (threadIdx.x < (ne ? 4 : 3)) {
        long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        add_counter(series_slot(g.ctrl, sweep) + threadIdx.x, s);
    }
    __syncthreads();
}

template <bool kNE>
__global__ void __launch_bounds__(kThreads) k_wide_half(Geom g, int colour, int off)
{
    __shared__ uint32_t sthr[16];
    __shared__ int red[kThreads / 32][4];
    if (threadIdx.x < 16) sthr[threadIdx.x] = g.thr16[threadIdx.x];
    __syncthreads();
    const unsigned long long sweep = g.ctrl->sweep + (unsigned long long)off;
    PhiloxPre pp;
    philox_prepare(pp, (uint32_t)sweep, (uint32_t)(sweep >> 32), g.key0, g.key1);
    const uint32_t cpr = g.half >> 4;  // 16-site chunks per plane row
    Counts cnt;
    const SweepView v = sweep_view(g);
    // Grid-stride over chunks with one resident wave of CTAs: the counter
    // reduction (and its barrier) happens once per CTA, not once per chunk.
    const uint64_t total = (uint64_t)g.L * cpr;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x)
        wide_chunk<kNE>(v, sthr, colour, sweep, pp, (int)(t / cpr), (int)(t % cpr), cnt);
    if (colour == 1) flush(v, sweep, cnt, kNE, red);
}

}  // namespace

bool wide_supported(const Geom &g)
{
    if (!(g.dims == 2 && g.two_S == 1 && g.bits[0] == nullptr && (g.L % 32) == 0)) return false;
    for (int k = 0; k < 16; ++k) {
        if ((k & 7) > 4) continue;
        if (!((g.always16 >> k) & 1u) && g.thr16[k] == 0u) return false;
    }
    return true;
}

int wide_chunks(const Geom &g) { return (int)(((uint64_t)g.L * (g.half >> 4) + kThreads - 1) / kThreads); }

cudaError_t launch_sweep_wide(const Geom &g, int off, cudaStream_t st)
{
    const Geom k = tiled_geom(g);  // compact table in t' = thr - 1 form
    // one wave: SMs x resident CTAs per SM (queried once per model)
    static int resident[2] = {0, 0};
    const int m = g.model == LAT_NE ? 1 : 0;
    if (resident[m] == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (m) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wide_half<true>, kThreads, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wide_half<false>, kThreads, 0);
        resident[m] = sms * (per > 0 ? per : 1);
    }
    const unsigned blocks = (unsigned)std::min<long long>(wide_chunks(g), resident[m]);
    for (int colour = 0; colour < 2; ++colour) {
        if (g.model == LAT_NE)
            k_wide_half<true><<<blocks, kThreads, 0, st>>>(k, colour, off);
        else
            k_wide_half<false><<<blocks, kThreads, 0, st>>>(k, colour, off);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lat
