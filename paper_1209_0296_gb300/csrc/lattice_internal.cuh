// lattice_internal.cuh -- device-side definitions shared by the library's
// kernels: Philox4x32-10, the per-lattice parameter block, the threshold
// table entry and warp/block reductions.  Library code only; the CPU
// oracle has its own independent copy of every rule.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.h"

#if defined(__CUDACC__)
#define LAT_HD __host__ __device__ __forceinline__
#define LAT_D __device__ __forceinline__
#else
#define LAT_HD inline
#define LAT_D inline
#endif

namespace lat {

// Philox4x32-10 of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of two
// 32x32 -> 64-bit multiplications by fixed odd constants, with the two key
// words advanced by the Weyl increments (golden ratio, sqrt(3)-1) between
// rounds.  Replaces the paper's per-thread LCG of §IV (Eqs. 5-7) so that a
// draw depends only on (seed, site group, sweep, colour).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct U4 {
    uint32_t x, y, z, w;
};

// 32 x 32 -> 64-bit product as one wide multiply (a single IMAD.WIDE on
// the GPU rather than a low and a high multiply).
LAT_HD void mul_hi_lo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

LAT_HD U4 philox(U4 c, uint32_t k0, uint32_t k1)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        mul_hi_lo(kPhiloxM0, c.x, h0, l0);
        mul_hi_lo(kPhiloxM1, c.z, h1, l1);
        U4 n;
        n.x = h1 ^ c.y ^ k0;
        n.y = l1;
        n.z = h0 ^ c.w ^ k1;
        n.w = l0;
        c = n;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// Philox4x32-10 for counters (g, c1, c2, c3) whose words 1..3 and key are
// fixed for a whole launch (sweep and colour): round 1's product of c2 and
// round 2's product of the round-1 word 0 do not depend on g, so they are
// computed once per thread; an item then costs 18 wide products and 19
// XORs.  Same rounds, constants and key schedule as philox() above.
struct PhiloxPre {
    uint32_t A, B;    // round-1 outputs 0 and 1
    uint32_t H2, L2;  // round-2 product of A: hi, lo
    uint32_t k0[10], k1[10];
};

LAT_HD void philox_prepare(PhiloxPre &pp, uint32_t ctr1, uint32_t ctr2, uint32_t key0, uint32_t key1)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        pp.k0[r] = key0 + (uint32_t)r * kPhiloxW0;
        pp.k1[r] = key1 + (uint32_t)r * kPhiloxW1;
    }
    uint32_t h1, l1;
    mul_hi_lo(kPhiloxM1, ctr2, h1, l1);
    pp.A = h1 ^ ctr1 ^ pp.k0[0];
    pp.B = l1;
    mul_hi_lo(kPhiloxM0, pp.A, pp.H2, pp.L2);
}

LAT_HD U4 philox_item(const PhiloxPre &pp, uint32_t g, uint32_t c3)
{
    uint32_t h0, l0, h1, l1;
    // round 1: (g, c1, c2, c3) -> (A, B, hi(M0 g) ^ c3 ^ k1, lo(M0 g))
    mul_hi_lo(kPhiloxM0, g, h0, l0);
    const uint32_t z1 = h0 ^ c3 ^ pp.k1[0];
    // round 2: (A, B, z1, l0) -> (hi(M1 z1) ^ B ^ k0, lo(M1 z1), H2 ^ l0 ^ k1, L2)
    mul_hi_lo(kPhiloxM1, z1, h1, l1);
    U4 c;
    c.x = h1 ^ pp.B ^ pp.k0[1];
    c.y = l1;
    c.z = pp.H2 ^ l0 ^ pp.k1[1];
    c.w = pp.L2;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 2; r < 10; ++r) {
        mul_hi_lo(kPhiloxM0, c.x, h0, l0);
        mul_hi_lo(kPhiloxM1, c.z, h1, l1);
        U4 n;
        n.x = h1 ^ c.y ^ pp.k0[r];
        n.y = l1;
        n.z = h0 ^ c.w ^ pp.k1[r];
        n.w = l0;
        c = n;
    }
    return c;
}

LAT_HD uint32_t word_of(const U4 &v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// One acceptance-table entry: accept without a draw (always = 1), or
// accept iff the 32-bit draw u < thr.
struct TabEntry {
    uint32_t thr;
    uint32_t always;
};

// Dynamic, device-resident state of one lattice: read by every sweep
// kernel so that a captured CUDA graph can be replayed unchanged.
struct Ctrl {
    unsigned long long sweep;        // global index of the next sweep
    unsigned long long *series;      // [series_cap][4] exact counters
    unsigned long long series_base;  // global sweep index of series[0]
    unsigned long long series_cap;   // sweeps the series buffer can hold
    unsigned long long *acf;         // [series_cap] sum_i s_i(t) s_i(ref), same indexing
    unsigned long long *fld;         // [series_cap] sum_i eta_i s_i (per-site field signs), same indexing
};

// Work items of the batched 8-site-chunk kernels (3D / spin-S, Potts): a
// band of plane rows x a segment of up to 256 chunk columns of one colour of
// one lattice.  A CTA of 256 threads covers rsb rows per pass (cpr chunks
// each) and `passes` passes per item, so an item is br = passes * rsb rows.
struct ColItemShape {
    uint32_t cpr, nseg, rsb, br;   // chunks per row, column segments, rows per pass, rows per band
};

// passes: rows a thread visits per item (batch_item_passes), or 0 for 8 on
// lattices of at least 2^16 chunks and 2 below.
LAT_HD ColItemShape col_item_shape(uint32_t half, uint32_t rows, uint32_t passes)
{
    ColItemShape sh;
    sh.cpr = half >> 3;
    sh.nseg = (sh.cpr + 255u) / 256u;
    sh.rsb = sh.cpr <= 256u ? 256u / sh.cpr : 1u;
    if (passes == 0u) passes = (uint64_t)rows * sh.cpr >= 65536u ? 8u : 2u;
    sh.br = passes * sh.rsb;
    return sh;
}

#if defined(__CUDACC__)
// Programmatic dependent launch.  The sweep kernels are launched so that the
// next kernel on the stream may be scheduled while this one drains.  Each
// calls dep_wait() before it touches anything an earlier kernel writes (the
// sweep counter, spins, flags, counters), and dep_launch() only when its own
// main work is done, so the successor's CTAs (which then sit in dep_wait())
// are placed on SMs no earlier than every CTA of this grid has run: when
// other streams' kernels share the GPU and not all of this grid fits at
// once, an earlier trigger could let waiting successor CTAs take the slots
// this grid's remaining CTAs need.  Launched without the attribute (or with
// no kernel before it), dep_wait() returns at once.
LAT_D void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
LAT_D void dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch kern<<<grid, block, 0, st>>>(args...) with programmatic stream
// serialisation (the kernel must call dep_wait() as above).
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), unsigned grid, unsigned block, cudaStream_t st, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<P>(args)...);
}

// Counter slot of global sweep `sweep` (4 x int64: bond, mag, up, unflipped).
LAT_D unsigned long long *series_slot(const Ctrl *c, unsigned long long sweep)
{
    return c->series + 4ull * (sweep - c->series_base);
}

// Autocorrelation slot of global sweep `sweep`: the overlap of the state
// after that sweep with the stored reference state (written only while a
// reference is set).
LAT_D unsigned long long *acf_slot(const Ctrl *c, unsigned long long sweep)
{
    return c->acf + (sweep - c->series_base);
}

// Field-sum slot of global sweep `sweep`: sum_i eta_i s_i over the state
// after that sweep (written by the kernels that read per-site disorder).
LAT_D unsigned long long *fld_slot(const Ctrl *c, unsigned long long sweep)
{
    return c->fld + (sweep - c->series_base);
}
#endif

// Static description of one lattice, passed by value to its kernels and
// stored in device memory for the batched engine.
struct Geom {
    int dims, L, two_S, model, cmode;
    int sh;               // log2(sites per Philox call)
    uint32_t G;           // Philox groups per row = ceil((L/2) >> sh)
    uint32_t rows;        // L^(dims-1)
    uint64_t N;           // sites
    uint32_t key0, key1;  // Philox key = seed
    int dsmax, nmax, nn, tab_n;
    const TabEntry *tab;  // [nds * nn], nds = 2*dsmax+1
    // Spins are double-buffered: after t sweeps the state is in s[t & 1]
    // (int8 layout) or bits[t & 1] (bit-packed layout).  A sweep reads one
    // buffer and writes the other, so no CTA can see a neighbour's
    // half-finished sweep.
    //
    // int8 layout is checkerboard-planar: plane c (colour c), row
    // r = y + L*z, index j = x >> 1 holds the spin at x = 2j + ((c+y+z)&1):
    //   s[buf][c * (N/2) + r * (L/2) + j].
    // Bit-packed layout: bits[buf][(c * L + y) * bw + (j >> 5)] bit (j & 31).
    int8_t *s[2];
    uint32_t *bits[2];
    uint32_t bw;          // bit-packed words per row
    uint32_t half;        // L/2: sites per plane row
    uint64_t plane;       // N/2: sites per plane
    // North-East persistence: one byte per Philox group of 4 same-colour
    // sites, bit q = site 4m+q ever changed: flags[(c * rows + r) * G + m].
    uint8_t *flags;
    // Reference state s(0) for the autocorrelation Phi(t) (§III.B, Eq. 4):
    // a copy in the int8 planar layout (ref) or the bit-packed one
    // (ref_bits); null when no reference is set.
    const int8_t *ref;
    const uint32_t *ref_bits;
    // Per-site disorder of Eq. 1 (J_ij = J * eps_ij, B_i = h * eta_i): one
    // byte per site in the int8 planar layout.  Bits 0..5 = the bonds to
    // x-1, x+1, y-1, y+1, z-1, z+1, set = that eps_ij is -1; bit 6 set =
    // eta_i is -1, whose acceptance entries sit in a second table half
    // (for -h) right after the first.  Null: uniform J and h.
    const uint8_t *cpl;
    Ctrl *ctrl;
    // Compact acceptance table for 2D spin-1/2 (tiled and bit-packed
    // kernels): index (self down) << 3 | (# down neighbours).
    uint32_t thr16[16];
    uint32_t always16;
    // 1 when no entry that a spin-1/2 or spin-1 move can reach is
    // never-accept (not always and thr = 0), so the table converts to the
    // t' = thr - 1 form of the byte-parallel 3D / spin-1 kernels.
    uint32_t tab_strict;
};

// The fields of a Geom that the 2D spin-1/2 sweep kernels read, small
// enough to live in registers (the batched kernels build it from a
// descriptor staged in shared memory).
struct SweepView {
    int L;
    uint32_t rows, half, G;
    uint64_t plane;
    int8_t *s0, *s1;
    uint32_t key0, key1;
    uint8_t *flags;
    const int8_t *ref;
    const uint8_t *cpl;
    Ctrl *ctrl;
};

LAT_HD SweepView sweep_view(const Geom &g)
{
    SweepView v;
    v.L = g.L;
    v.rows = g.rows;
    v.half = g.half;
    v.G = g.G;
    v.plane = g.plane;
    v.s0 = g.s[0];
    v.s1 = g.s[1];
    v.key0 = g.key0;
    v.key1 = g.key1;
    v.flags = g.flags;
    v.ref = g.ref;
    v.cpl = g.cpl;
    v.ctrl = g.ctrl;
    return v;
}

// Planar address of site (x, y, z) (coordinates already wrapped).
LAT_HD uint64_t planar_index(const Geom &g, int x, int y, int z)
{
    const int c = (x + y + z) & 1;
    const uint64_t r = (uint64_t)y + (uint64_t)g.L * (uint64_t)z;
    return (uint64_t)c * g.plane + r * g.half + (uint64_t)(x >> 1);
}

// w mod n for w < 2n (a neighbour word index one step past either row end).
LAT_HD uint32_t wrap_once(uint32_t w, uint32_t n) { return w >= n ? w - n : w; }

// Spin value <-> state index (state 0 = most negative value).
LAT_HD int spin_of_state(int two_S, int k) { return (two_S & 1) ? 2 * k - two_S : k - (two_S >> 1); }
LAT_HD int state_of_spin(int two_S, int s) { return (two_S & 1) ? (s + two_S) >> 1 : s + (two_S >> 1); }
LAT_HD int max_spin(int two_S) { return (two_S & 1) ? two_S : (two_S >> 1); }

#if defined(__CUDACC__)
// Sum of an int over the block; result valid in thread 0.  `red` must hold
// one int per warp.  Every thread of the block must call it.
LAT_D long long block_sum_ll(long long v, long long *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) t += red[w];
    }
    return t;
}

LAT_D void add_counter(unsigned long long *slot, long long v)
{
    if (v != 0) atomicAdd(slot, (unsigned long long)v);
}
#endif

}  // namespace lat

// Host-side launchers implemented in the .cu files.
namespace lat {
cudaError_t launch_init(const Geom &g, int init, double c, cudaStream_t st);
cudaError_t launch_half_sweep_generic(const Geom &g, int colour, int off, cudaStream_t st);
// out[0..4] += bond, mag, up, unflipped, field sum (sum_i eta_i s_i)
cudaError_t launch_measure(const Geom &g, const int8_t *spins, unsigned long long *out5, cudaStream_t st);
cudaError_t launch_advance(Ctrl *ctrl, unsigned long long k, cudaStream_t st);
cudaError_t launch_set_ctrl(Ctrl *ctrl, unsigned long long sweep, unsigned long long *series,
                            unsigned long long base, unsigned long long cap, unsigned long long *acf,
                            unsigned long long *fld, cudaStream_t st);
bool tiled_supported(const Geom &g);
cudaError_t launch_sweep_tiled(const Geom &g, int tile_w, int tile_h, int off, cudaStream_t st);
cudaError_t launch_pack_bits(const Geom &g, const int8_t *planar, uint32_t *bits, cudaStream_t st);
cudaError_t launch_unpack_bits(const Geom &g, const uint32_t *bits, int8_t *planar, cudaStream_t st);
// planar <-> x-fastest (linear) int8 spins
cudaError_t launch_to_linear(const Geom &g, const int8_t *planar, int8_t *linear, cudaStream_t st);
// out[0] += number of bytes of spins[0 .. N) that are not allowed values.
cudaError_t launch_count_bad(const Geom &g, const int8_t *spins, unsigned long long *out, cudaStream_t st);
cudaError_t launch_to_planar(const Geom &g, const int8_t *linear, int8_t *planar, cudaStream_t st);
cudaError_t launch_sweep_bitpacked(const Geom &g, int off, cudaStream_t st);
bool bitpacked_supported(const Geom &g);
bool wide_supported(const Geom &g);
// fields: per-site field signs are set (g.cpl bit 6; the -h table half
// follows the first in g.tab, with no never-accept entry)
cudaError_t launch_sweep_wide(const Geom &g, bool fields, int off, cudaStream_t st);
// The paper's random-sub-lattice, random-site sweep (kernels_rsite.cu).
// balanced: the balance-preserving variant (single-colour rounds, four launches)
bool rsite_params_ok(const Geom &g, int b, int lambda, bool balanced);
cudaError_t launch_sweep_rsite(const Geom &g, int8_t *scratch, int b, int lambda, bool balanced, int off,
                               cudaStream_t st);
bool resident_supported(const Geom &g);
cudaError_t launch_sweep_resident(const Geom &g, int off, int n_sweeps, cudaStream_t st);
size_t resident_smem_bytes(const Geom &g);
// geoms: compact-table descriptors (tiled_geom); n[i]: sweeps for lattice i
cudaError_t launch_batch_resident(const Geom *geoms, const long long *n, int n_lat, long long done, int chunk,
                                  size_t smem, cudaStream_t st);
bool wide3_supported(const Geom &g);
// q-state Potts model, 8 sites per thread (kernels_potts.cu)
bool potts_supported(const Geom &g);
cudaError_t launch_sweep_potts(const Geom &g, int off, cudaStream_t st);
// batch items of one colour of one lattice; passes: rows a thread visits per item
int potts_items(const Geom &g, int passes);
int batch_potts_grid();
cudaError_t launch_batch_potts(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int colour, int passes, int grid, cudaStream_t st);
cudaError_t launch_sweep_wide3(const Geom &g, int off, cudaStream_t st);
// the byte-parallel step applies (spin-1/2 or spin-1, strict table)
bool wide3_swar(const Geom &g);
// batch items of one colour of one lattice; passes: rows a thread visits
// per item (0: the size-based default)
int wide3_items(const Geom &g, int passes);
// rows per thread of the 3D / spin-S or Potts items of a phase with
// chunk_rows (row, chunk) pairs of that kind
int batch_item_passes(uint64_t chunk_rows);
int batch_wide3_grid(bool swar);
cudaError_t launch_batch_wide3(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int colour, bool swar, int passes, int grid, cudaStream_t st);
int wide_chunks(const Geom &g);
// 2D spin-1/2 Ising / North-East with uniform couplings at any even L (the
// wide kernel's sweep on rows at any byte alignment; launch_sweep_wide takes
// these lattices when L % 32 != 0), and its batched form
bool any_supported(const Geom &g);
// batch items of one colour of one lattice; passes: rows a thread visits
// per item (0: the size-based default)
int any_items(const Geom &g, int passes);
int batch_any_grid(bool ne);
// aligned: every lattice of the items has L % 32 == 0 (16-byte aligned
// rows); cmode (with ne): every lattice of the items is a c-mode North-East one
cudaError_t launch_batch_any(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item, int colour,
                             bool ne, bool cmode, bool aligned, int passes, int grid, cudaStream_t st);
// batched engine
Geom tiled_geom(const Geom &g);
int tiles_of(const Geom &g, int tile_h);
int batch_tiled_grid(bool ne);
cudaError_t launch_batch_tiled(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                               int tile_h, int off, int grid, bool ne, cudaStream_t st);
// tab_max: the largest tab_n among the lattices of the items
cudaError_t launch_batch_generic(const Geom *geoms, const uint2 *items, int n_items, unsigned *next_item,
                                 int colour, int off, int grid, int tab_max, cudaStream_t st);
int batch_generic_grid();
cudaError_t launch_batch_advance(Ctrl *const *ctrls, int n, unsigned *counters, int n_counters,
                                 unsigned long long k, cudaStream_t st);
}  // namespace lat
