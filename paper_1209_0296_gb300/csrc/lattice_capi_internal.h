// lattice_capi_internal.h -- host-side handle of one lattice and helpers
// shared by the C-ABI, batch and server translation units.
#pragma once

#include <atomic>
#include <string>
#include <vector>

#include "lattice_internal.cuh"

namespace lat {

struct Params {
    int dims, L, two_S, model, cmode, init, layout;
    double J, h, T, c;
    uint64_t seed;
    uint64_t N;
};

int cuda_fail(cudaError_t e, const char *what);
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);
int validate(int dims, int L, int two_S, int model, double J, double h, double T_or_c, int init,
             int layout, Params &P);
void build_table(const Params &P, std::vector<TabEntry> &tab, int &dsmax, int &nmax, int &nn);
size_t footprint_bytes(const Params &P);
int create_impl(struct ::lattice **out, int dims, int L, int two_S, int model, double J, double h,
                double T_or_c, uint64_t seed, int init, int layout, void *cuda_stream);
int sweep_impl(struct ::lattice *lt, int64_t n);
int choose_kernel(const struct ::lattice *lt);
int ensure_series(struct ::lattice *lt, unsigned long long need);
bool tile_shape_ok(int tile_w, int tile_h);
int default_tile_h();
void compact_table(Geom &g, const TabEntry *host_tab);

// Sweeps per captured CUDA graph: small lattices are launch-bound, so they
// replay long graphs; large ones need only a few sweeps per graph.
inline int default_graph_sweeps(const Params &P)
{
    if (P.N <= (1u << 16)) return 64;
    if (P.N <= (1u << 22)) return 16;
    return 8;
}

}  // namespace lat

struct lattice {
    lat::Params P;
    lat::Geom geom;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int8_t *spins[2] = {nullptr, nullptr};   // int8 layout: double buffer; bit-packed: [0] = staging
    uint8_t *flags = nullptr;      // North-East persistence bytes (see Geom)
    uint32_t *bits[2] = {nullptr, nullptr};
    lat::TabEntry *tab = nullptr;
    lat::Ctrl *ctrl = nullptr;
    // [series_cap][4] counters, then [series_cap] overlaps, then [series_cap] field sums
    unsigned long long *series = nullptr;
    unsigned long long series_cap = 0;   // sweeps the buffer can hold (from series_first)
    int8_t *ref = nullptr;               // reference state s(0), int8 planar layout
    uint32_t *ref_bits = nullptr;        // reference state s(0), bit-packed layout
    int64_t ref_sweep = -1;              // sweeps done when the reference was taken (-1: none)
    int dynamics = 0;                    // LAT_DYNAMICS_*
    int rs_tile = 0, rs_lambda = 0;      // random-site sub-lattice side and picks per round
    int8_t *rs_scratch = nullptr;        // random-site: output of the first launch of a sweep
    uint8_t *cpl = nullptr;              // per-site disorder bytes (see Geom::cpl); null when all zero
    std::vector<uint8_t> dis_host;       // host copy of the disorder bytes (empty: none set)
    bool has_bonds = false;              // coupling signs set
    bool has_fields = false;             // field signs set (the table then has a -h half)
    bool fields_wide_ok = false;         // the -h half suits the 2D wide kernel
    int64_t disorder_from = 0;           // sweeps done when the couplings or field signs last changed
    int64_t fields_from = 0;             // sweeps done when the field signs were last set
    unsigned long long *scratch4 = nullptr;
    std::vector<lat::TabEntry> host_tab;
    int64_t sweeps = 0;        // sweeps done (global index of the next sweep)
    int64_t series_first = 0;  // first sweep index recorded in the series buffer
    int kernel = 0, tile_w = 0, tile_h = 0, graph_sweeps = 0;
    int tuned_kernel = 0;      // autotuner's choice for LAT_KERNEL_AUTO (0 = not tuned)
    bool graph_pinned = false; // sweeps per graph set by lattice_set_kernel (the tuner keeps it)
    cudaGraphExec_t graph_exec = nullptr;
    bool graph_valid = false;
};
