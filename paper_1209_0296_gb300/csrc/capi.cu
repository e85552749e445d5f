// capi.cu -- the C ABI of include/lattice.h for single lattices: argument
// checks, device memory, the host-built acceptance table, the sweep loop
// (direct launches or CUDA-graph replays), counters, checkpoints.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lattice_capi_internal.h"

namespace lat {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    g_last_cuda_error = buf;
    return LAT_ECUDA;
}

// Test hook: make the n-th next device allocation fail (0 = off).
static std::atomic<int> g_fail_alloc_countdown{0};

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st)
{
    int c = g_fail_alloc_countdown.load();
    if (c > 0) {
        if (g_fail_alloc_countdown.fetch_sub(1) == 1) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMallocAsync(p, bytes, st);
}

void dev_free(void *p, cudaStream_t st)
{
    if (p != nullptr) cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------------------
// Acceptance table (§III.A: P_acc = min[1, exp(-dH/T)]; §III.B: rates at
// concentration c).  Built on the host in double precision:
//   dE = -(J * (ds*n)) - h * ds
//   dE <= 0           -> always
//   otherwise         -> thr = floor(exp(-dE/T) * 2^32)
// North-East c-mode: p = c/(1-c) for ds > 0 (down->up), (1-c)/c for ds < 0;
// p >= 1 -> always, else thr = floor(p * 2^32).
// ---------------------------------------------------------------------------
void build_table(const Params &P, std::vector<TabEntry> &tab, int &dsmax, int &nmax, int &nn)
{
    if (P.model == LAT_POTTS) {
        // Potts: index (df + 1) * nn + (dn + nmax) with dn the change in the
        // number of equal neighbours (|dn| <= 2*dims) and df the change in
        // the state-0 indicator; dE = -(J*dn) - h*df.
        dsmax = 1;
        nmax = 2 * P.dims;
        nn = 2 * nmax + 1;
        tab.assign((size_t)3 * nn, TabEntry{0u, 0u});
        for (int df = -1; df <= 1; ++df)
            for (int dn = -nmax; dn <= nmax; ++dn) {
                const double dE = -(P.J * (double)dn) - P.h * (double)df;
                TabEntry e{0u, 0u};
                if (dE <= 0.0) e.always = 1u;
                else e.thr = (uint32_t)std::floor(std::ldexp(std::exp(-dE / P.T), 32));
                tab[(size_t)(df + 1) * nn + (dn + nmax)] = e;
            }
        return;
    }
    const int smax = max_spin(P.two_S);
    dsmax = 2 * smax;
    nmax = 2 * P.dims * smax;
    nn = 2 * nmax + 1;
    const int nds = 2 * dsmax + 1;
    tab.assign((size_t)nds * nn, TabEntry{0u, 0u});
    for (int ds = -dsmax; ds <= dsmax; ++ds) {
        for (int n = -nmax; n <= nmax; ++n) {
            TabEntry e{0u, 0u};
            double p;
            bool always;
            if (P.cmode) {
                p = ds > 0 ? P.c / (1.0 - P.c) : (1.0 - P.c) / P.c;
                always = (p >= 1.0);
            } else {
                const double dE = -(P.J * (double)(ds * n)) - P.h * (double)ds;
                always = (dE <= 0.0);
                p = always ? 1.0 : std::exp(-dE / P.T);
            }
            if (always) {
                e.always = 1u;
            } else {
                e.thr = (uint32_t)std::floor(std::ldexp(p, 32));
            }
            tab[(size_t)(ds + dsmax) * nn + (n + nmax)] = e;
        }
    }
}

int validate(int dims, int L, int two_S, int model, double J, double h, double T_or_c,
             int init, int layout, Params &P)
{
    if (dims != 2 && dims != 3) return LAT_EINVAL;
    if (L < 2 || (L & 1)) return LAT_EINVAL;
    if (two_S < 1 || two_S > 8) return LAT_EINVAL;
    if (model != LAT_ISING && model != LAT_NE && model != LAT_POTTS) return LAT_EINVAL;
    if (model == LAT_NE && (dims != 2 || two_S != 1)) return LAT_EINVAL;
    if (!std::isfinite(J) || !std::isfinite(h) || !std::isfinite(T_or_c)) return LAT_EINVAL;
    const double N = std::pow((double)L, (double)dims);
    if (N >= 4294967296.0) return LAT_EINVAL;
    const bool cmode = (model == LAT_NE && J == 0.0 && h == 0.0);
    if (cmode) {
        if (!(T_or_c > 0.0 && T_or_c < 1.0)) return LAT_EINVAL;
    } else if (!(T_or_c > 0.0)) {
        return LAT_EINVAL;
    }
    if (init != LAT_INIT_COLD && init != LAT_INIT_RANDOM && init != LAT_INIT_EQUILIBRIUM)
        return LAT_EINVAL;
    if (init == LAT_INIT_EQUILIBRIUM && !cmode) return LAT_EINVAL;
    if (layout != LAT_INT8 && layout != LAT_BITPACKED) return LAT_EINVAL;
    if (layout == LAT_BITPACKED && (dims != 2 || two_S != 1 || model == LAT_POTTS)) return LAT_ENOTSUP;
    P.dims = dims;
    P.L = L;
    P.two_S = two_S;
    P.model = model;
    P.J = J;
    P.h = h;
    P.cmode = cmode ? 1 : 0;
    P.T = cmode ? 0.0 : T_or_c;
    P.c = cmode ? T_or_c : 0.0;
    P.init = init;
    P.layout = layout;
    P.N = (uint64_t)N;
    return LAT_OK;
}

// Persistence flags: one byte per Philox group of same-colour sites.
static size_t flag_bytes(const Params &P)
{
    const size_t rows = (size_t)(P.dims == 3 ? (size_t)P.L * P.L : (size_t)P.L);
    const int sh = (P.two_S == 1) ? 2 : 1;
    const size_t G = ((size_t)(P.L / 2) + (1u << sh) - 1) >> sh;
    return 2 * rows * G;
}

// Bit-packed layout: two colour planes of L rows of bw words.
static size_t bits_bytes(const Params &P) { return (size_t)2 * P.L * (((size_t)P.L / 2 + 31) / 32) * 4; }

size_t footprint_bytes(const Params &P)
{
    size_t b = 2 * (size_t)P.N;                             // int8 spins, double-buffered
    if (P.model == LAT_NE) b += flag_bytes(P);              // persistence bytes
    if (P.layout == LAT_BITPACKED) b += (size_t)2 * P.L * (((size_t)P.L / 2 + 31) / 32) * 4;
    const int smax = max_spin(P.two_S);
    b += (size_t)(4 * smax + 1) * (4 * P.dims * smax + 1) * sizeof(TabEntry);
    b += sizeof(Ctrl) + 4096;                               // control + first series block
    return b;
}

// Make the per-sweep counter buffer hold global sweeps [series_first, need).
int ensure_series(lattice *lt, unsigned long long need)
{
    const unsigned long long base = (unsigned long long)lt->series_first;
    const unsigned long long slots = need > base ? need - base : 0;
    if (slots <= lt->series_cap && lt->series != nullptr) return LAT_OK;
    unsigned long long cap = lt->series_cap ? lt->series_cap : 64;
    while (cap < slots) cap *= 2;
    // [cap][4] counters, then [cap] reference overlaps (the autocorrelation),
    // then [cap] field sums
    const size_t bytes = (size_t)cap * 6 * sizeof(unsigned long long);
    void *p = nullptr;
    cudaError_t e = dev_alloc(&p, bytes, lt->stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "series alloc");
    unsigned long long *np = (unsigned long long *)p;
    e = cudaMemsetAsync(p, 0, bytes, lt->stream);
    if (e == cudaSuccess && lt->series != nullptr)
        e = cudaMemcpyAsync(np, lt->series, (size_t)lt->series_cap * 4 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, lt->stream);
    for (int sec = 4; sec < 6 && e == cudaSuccess && lt->series != nullptr; ++sec)
        e = cudaMemcpyAsync(np + sec * cap, lt->series + sec * lt->series_cap,
                            (size_t)lt->series_cap * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                            lt->stream);
    if (e == cudaSuccess)
        e = launch_set_ctrl(lt->ctrl, (unsigned long long)lt->sweeps, np, base, cap, np + 4 * cap, np + 5 * cap,
                            lt->stream);
    if (e != cudaSuccess) {
        dev_free(p, lt->stream);
        return cuda_fail(e, "series grow");
    }
    dev_free(lt->series, lt->stream);
    lt->series = (unsigned long long *)p;
    lt->series_cap = cap;
    return LAT_OK;
}

// Compact 16-entry table for spin-1/2 in 2D: index (sd << 3) | nd with sd = 1
// for a down spin (s = -1) and nd the number of down neighbours; then
// ds = s' - s = +2 (down->up) or -2, and n = 4 - 2*nd.
void compact_table(Geom &g, const TabEntry *host_tab)
{
    g.always16 = 0;
    for (int k = 0; k < 16; ++k) g.thr16[k] = 0;
    // the rows a spin-1/2 (ds = +-2) or spin-1 (ds = +-1, +-2) move reaches
    g.tab_strict = 0;
    if (g.two_S <= 2 && g.dsmax == 2) {
        g.tab_strict = 1;
        for (int ds = -2; ds <= 2; ++ds) {
            if (ds == 0 || (g.two_S == 1 && (ds & 1))) continue;
            for (int n = 0; n < g.nn; ++n) {
                const TabEntry e = host_tab[(ds + g.dsmax) * g.nn + n];
                if (!e.always && e.thr == 0u) g.tab_strict = 0;
            }
        }
    }
    if (g.dims != 2 || g.two_S != 1) return;
    for (int k = 0; k < 16; ++k) {
        const int sd = k >> 3, nd = k & 7;
        if (nd > 4) continue;
        const int ds = sd ? 2 : -2;
        const int n = 4 - 2 * nd;
        const TabEntry e = host_tab[(ds + g.dsmax) * g.nn + (n + g.nmax)];
        g.thr16[k] = e.thr;
        if (e.always) g.always16 |= 1u << k;
    }
}

// LAT_KERNEL_WIDE covers four kernels: the 2D spin-1/2 one for L % 32 == 0
// and its any-even-L form (kernels_wide.cu), the
// 3D / spin-S Ising one (kernels_wide3.cu) and the Potts one
// (kernels_potts.cu).
static bool wide2_supported(const Geom &g) { return wide_supported(g) || any_supported(g); }
static bool any_wide(const Geom &g) { return wide2_supported(g) || wide3_supported(g) || potts_supported(g); }

int choose_kernel(const lattice *lt)
{
    if (lt->P.layout == LAT_BITPACKED) return LAT_KERNEL_AUTO;  // bit-packed path
    if (lt->geom.cpl != nullptr)   // per-site disorder: the 2D wide kernel or the generic one
        return (lt->kernel != LAT_KERNEL_GENERIC && wide_supported(lt->geom) &&
                (!lt->has_fields || lt->fields_wide_ok))
                   ? LAT_KERNEL_WIDE
                   : LAT_KERNEL_GENERIC;
    if (lt->kernel == LAT_KERNEL_GENERIC) return LAT_KERNEL_GENERIC;
    if (lt->kernel == LAT_KERNEL_TILED && tiled_supported(lt->geom)) return LAT_KERNEL_TILED;
    if (lt->kernel == LAT_KERNEL_WIDE && any_wide(lt->geom)) return LAT_KERNEL_WIDE;
    if (lt->kernel == LAT_KERNEL_RESIDENT && resident_supported(lt->geom)) return LAT_KERNEL_RESIDENT;
    if (lt->kernel == LAT_KERNEL_AUTO && lt->tuned_kernel != 0) return lt->tuned_kernel;
    if (any_wide(lt->geom)) return LAT_KERNEL_WIDE;
    if (tiled_supported(lt->geom)) return LAT_KERNEL_TILED;
    return LAT_KERNEL_GENERIC;
}

// Queue k sweeps with sweep offsets 0..k-1 relative to ctrl->sweep, then
// advance ctrl->sweep by k.  Used directly and under stream capture.
// Sweeps per resident launch (a launch runs about a microsecond per sweep at
// L = 64, so this bounds one kernel to well under a second).
constexpr int64_t kResidentChunk = 1 << 16;

int enqueue_sweeps(lattice *lt, int64_t k, cudaStream_t st)
{
    if (lt->dynamics != LAT_DYNAMICS_CHECKERBOARD) {
        const bool balanced = lt->dynamics == LAT_DYNAMICS_RANDOM_SITE_BALANCED;
        for (int64_t off = 0; off < k; ++off) {
            cudaError_t e =
                launch_sweep_rsite(lt->geom, lt->rs_scratch, lt->rs_tile, lt->rs_lambda, balanced, (int)off, st);
            if (e != cudaSuccess) return cuda_fail(e, "random-site sweep launch");
        }
        cudaError_t e = launch_advance(lt->ctrl, (unsigned long long)k, st);
        if (e != cudaSuccess) return cuda_fail(e, "advance launch");
        return LAT_OK;
    }
    const int kern = choose_kernel(lt);
    if (kern == LAT_KERNEL_RESIDENT) {
        for (int64_t off = 0; off < k; off += kResidentChunk) {
            const int m = (int)std::min<int64_t>(kResidentChunk, k - off);
            cudaError_t e = launch_sweep_resident(lt->geom, (int)off, m, st);
            if (e != cudaSuccess) return cuda_fail(e, "resident sweep launch");
        }
        cudaError_t e = launch_advance(lt->ctrl, (unsigned long long)k, st);
        if (e != cudaSuccess) return cuda_fail(e, "advance launch");
        return LAT_OK;
    }
    for (int off = 0; off < k; ++off) {
        cudaError_t e;
        if (lt->P.layout == LAT_BITPACKED) {
            e = launch_sweep_bitpacked(lt->geom, off, st);
        } else if (kern == LAT_KERNEL_TILED) {
            e = launch_sweep_tiled(lt->geom, lt->tile_w, lt->tile_h, off, st);
        } else if (kern == LAT_KERNEL_WIDE) {
            e = wide2_supported(lt->geom)   ? launch_sweep_wide(lt->geom, lt->has_fields, off, st)
                : potts_supported(lt->geom) ? launch_sweep_potts(lt->geom, off, st)
                                            : launch_sweep_wide3(lt->geom, off, st);
        } else {
            e = launch_half_sweep_generic(lt->geom, 0, off, st);
            if (e == cudaSuccess) e = launch_half_sweep_generic(lt->geom, 1, off, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    }
    cudaError_t e = launch_advance(lt->ctrl, (unsigned long long)k, st);
    if (e != cudaSuccess) return cuda_fail(e, "advance launch");
    return LAT_OK;
}

static int ensure_graph(lattice *lt)
{
    if (lt->graph_valid) return LAT_OK;
    if (lt->graph_exec != nullptr) {
        cudaGraphExecDestroy(lt->graph_exec);
        lt->graph_exec = nullptr;
    }
    if (lt->cap_stream == nullptr) {
        cudaError_t e = cudaStreamCreateWithFlags(&lt->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(lt->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int rc = enqueue_sweeps(lt, lt->graph_sweeps, lt->cap_stream);
    e = cudaStreamEndCapture(lt->cap_stream, &graph);
    if (rc != LAT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&lt->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    lt->graph_valid = true;
    return LAT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner for LAT_KERNEL_AUTO: the first sweep call with enough sweeps
// times candidates on the caller's own sweeps and keeps the fastest.
//  1. The kernel, when the lattice has more than one candidate (2D spin-1/2
//     with L % 32 == 0: the wide two-launch kernel, the tiled one-launch
//     kernel at two tile heights and, when the lattice fits one CTA, the
//     resident kernel).
//  2. The sweeps per CUDA-graph replay, for every lattice the sweep loop
//     runs through graphs (any dims, spin and model): half, one, two and
//     four times the default size, as far as the call's sweeps reach.
// Each candidate is timed the way the sweep loop will run it: the resident
// kernel as one launch, the others as a replayed CUDA graph after one
// untimed replay, so launch overheads count as they will.  Every kernel and
// graph size produces the same bits, so tuning changes no result.  Choices
// are cached per (model, dims, 2S, L) for the life of the process and, when
// LATTICE_TUNE_CACHE names a file, across processes: one JSON object per
// line, {"model": m, "dims": d, "two_S": s, "L": L, "kernel": k,
// "tile_h": h, "graph": g}, read before the first lookup and appended to
// after each new tuning (a line of the older form {"model", "L", "kernel",
// "tile_h"} reads as a 2D spin-1/2 lattice with the default graph size).
// An entry the lattice cannot run (a hand-edited file) is ignored.
// ---------------------------------------------------------------------------
namespace {
struct TuneChoice {
    int kernel, tile_h, graph;   // graph: sweeps per replay, 0 = the default
};
using TuneKey = std::tuple<int, int, int, int>;   // model, dims, two_S, L
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;
bool g_tune_file_read = false;
constexpr int kTuneSweeps = 4;

TuneKey tune_key(const lattice *lt) { return TuneKey(lt->P.model, lt->P.dims, lt->P.two_S, lt->P.L); }

const char *tune_cache_path()
{
    const char *p = std::getenv("LATTICE_TUNE_CACHE");
    return (p != nullptr && *p != '\0') ? p : nullptr;
}

// With g_tune_mu held: merge the cache file's entries (once per process).
void read_tune_file()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = tune_cache_path();
    if (path == nullptr) return;
    FILE *f = std::fopen(path, "r");
    if (f == nullptr) return;
    char line[512];
    while (std::fgets(line, sizeof line, f) != nullptr) {
        int m = 0, d = 0, s2 = 0, L = 0, k = 0, h = 0, gs = 0;
        if (std::sscanf(line,
                        " {\"model\": %d, \"dims\": %d, \"two_S\": %d, \"L\": %d, \"kernel\": %d, \"tile_h\": %d, "
                        "\"graph\": %d}",
                        &m, &d, &s2, &L, &k, &h, &gs) == 7)
            g_tune[TuneKey(m, d, s2, L)] = TuneChoice{k, h, gs};
        else if (std::sscanf(line, " {\"model\": %d, \"L\": %d, \"kernel\": %d, \"tile_h\": %d}", &m, &L, &k, &h) ==
                 4)
            g_tune[TuneKey(m, 2, 1, L)] = TuneChoice{k, h, 0};
    }
    std::fclose(f);
}

// With g_tune_mu held: append one tuned choice to the cache file.
void append_tune_file(const TuneKey &key, const TuneChoice &c)
{
    const char *path = tune_cache_path();
    if (path == nullptr) return;
    FILE *f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f,
                 "{\"model\": %d, \"dims\": %d, \"two_S\": %d, \"L\": %d, \"kernel\": %d, \"tile_h\": %d, "
                 "\"graph\": %d}\n",
                 std::get<0>(key), std::get<1>(key), std::get<2>(key), std::get<3>(key), c.kernel, c.tile_h, c.graph);
    std::fclose(f);
}

// Whether a choice runs on this lattice.
bool tune_choice_ok(const lattice *lt, const TuneChoice &c)
{
    if (c.graph < 0 || c.graph > 4096) return false;
    switch (c.kernel) {
    case LAT_KERNEL_WIDE: return any_wide(lt->geom);
    case LAT_KERNEL_TILED: return tiled_supported(lt->geom) && tile_shape_ok(0, c.tile_h);
    case LAT_KERNEL_RESIDENT: return resident_supported(lt->geom);
    case LAT_KERNEL_GENERIC: return true;
    default: return false;
    }
}

// Time one replay of a graph of n sweeps after one untimed replay (the
// resident kernel: two launches of n sweeps, the second timed); 2n sweeps
// are enqueued on the lattice's stream.
int time_candidate(lattice *lt, int n, cudaEvent_t ev0, cudaEvent_t ev1, float &ms)
{
    cudaGraphExec_t exec = nullptr;
    int rc = LAT_OK;
    const bool graphed = choose_kernel(lt) != LAT_KERNEL_RESIDENT;
    if (graphed) {
        if (lt->cap_stream == nullptr &&
            cudaStreamCreateWithFlags(&lt->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return LAT_ECUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(lt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return LAT_ECUDA;
        rc = enqueue_sweeps(lt, n, lt->cap_stream);
        const cudaError_t e = cudaStreamEndCapture(lt->cap_stream, &graph);
        if (rc == LAT_OK && e != cudaSuccess) rc = LAT_ECUDA;
        if (rc == LAT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = LAT_ECUDA;
        if (graph) cudaGraphDestroy(graph);
        if (rc != LAT_OK) return rc;
    }
    for (int rep = 0; rep < 2 && rc == LAT_OK; ++rep) {
        if (rep == 1 && cudaEventRecord(ev0, lt->stream) != cudaSuccess) rc = LAT_ECUDA;
        if (rc == LAT_OK) {
            if (graphed) rc = cudaGraphLaunch(exec, lt->stream) == cudaSuccess ? LAT_OK : LAT_ECUDA;
            else rc = enqueue_sweeps(lt, n, lt->stream);
        }
    }
    if (rc == LAT_OK && cudaEventRecord(ev1, lt->stream) != cudaSuccess) rc = LAT_ECUDA;
    if (rc == LAT_OK && cudaEventSynchronize(ev1) != cudaSuccess) rc = LAT_ECUDA;
    if (rc == LAT_OK && cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) rc = LAT_ECUDA;
    if (exec) cudaGraphExecDestroy(exec);
    if (rc == LAT_ECUDA) return cuda_fail(cudaGetLastError(), "autotune");
    return rc;
}

// Apply a choice to the lattice (the user's own tile or graph size wins).
void apply_choice(lattice *lt, const TuneChoice &c)
{
    lt->tuned_kernel = c.kernel;
    if (lt->tile_h == 0) lt->tile_h = c.tile_h;
    if (!lt->graph_pinned && c.graph > 0) lt->graph_sweeps = c.graph;
    lt->graph_valid = false;
}
}  // namespace

static int autotune(lattice *lt, int64_t &left)
{
    const TuneKey key = tune_key(lt);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        read_tune_file();
        auto it = g_tune.find(key);
        if (it != g_tune.end() && tune_choice_ok(lt, it->second)) {
            apply_choice(lt, it->second);
            return LAT_OK;
        }
    }
    // kernel candidates
    std::vector<TuneChoice> cand;
    const bool d2 = lt->P.dims == 2 && lt->P.two_S == 1 && lt->P.model != LAT_POTTS;
    if (any_wide(lt->geom)) cand.push_back(TuneChoice{LAT_KERNEL_WIDE, 0, 0});
    if (d2 && tiled_supported(lt->geom)) {
        cand.push_back(TuneChoice{LAT_KERNEL_TILED, 64, 0});
        cand.push_back(TuneChoice{LAT_KERNEL_TILED, 32, 0});
    }
    if (d2 && resident_supported(lt->geom)) cand.push_back(TuneChoice{LAT_KERNEL_RESIDENT, 0, 0});
    if (cand.empty()) cand.push_back(TuneChoice{LAT_KERNEL_GENERIC, 0, 0});
    const int n_c = (int)cand.size();
    const int g0 = default_graph_sweeps(lt->P);
    // too short to tune now (a later, longer call tunes): the kernel when
    // there is a choice, else at least the smallest graph size
    if (n_c > 1 && left < (int64_t)(n_c * 2 * kTuneSweeps)) return LAT_OK;
    if (n_c == 1 && (lt->graph_pinned || cand[0].kernel == LAT_KERNEL_RESIDENT || left < 2 * (int64_t)std::max(2, g0 / 2)))
        return LAT_OK;
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return LAT_OK;
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return LAT_OK;
    }
    const int keep_tile = lt->tile_h;
    const int keep_graph = lt->graph_sweeps;
    TuneChoice pick = cand[0];
    int rc = LAT_OK;
    if (n_c > 1) {
        float best = 1e30f;
        for (int c = 0; c < n_c && rc == LAT_OK; ++c) {
            lt->tuned_kernel = cand[(size_t)c].kernel;
            lt->tile_h = cand[(size_t)c].tile_h;
            float ms = 0.f;
            rc = time_candidate(lt, kTuneSweeps, ev[0], ev[1], ms);
            if (rc != LAT_OK) break;
            lt->sweeps += 2 * kTuneSweeps;
            left -= 2 * kTuneSweeps;
            if (ms < best) {
                best = ms;
                pick = cand[(size_t)c];
            }
        }
    }
    lt->tuned_kernel = pick.kernel;
    lt->tile_h = keep_tile ? keep_tile : pick.tile_h;
    // sweeps per graph replay (graph-launched kernels, size not set by the user)
    if (rc == LAT_OK && pick.kernel != LAT_KERNEL_RESIDENT && !lt->graph_pinned) {
        float best = 1e30f;
        for (int f : {1, 2, 4, 8}) {   // g0 / 2, g0, 2 g0, 4 g0
            const int gs = std::max(2, g0 * f / 2);
            if (left < 2 * (int64_t)gs) break;
            float ms = 0.f;
            rc = time_candidate(lt, gs, ev[0], ev[1], ms);
            if (rc != LAT_OK) break;
            lt->sweeps += 2 * gs;
            left -= 2 * gs;
            if (ms / gs < best) {
                best = ms / gs;
                pick.graph = gs;
            }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    lt->graph_sweeps = keep_graph;
    if (rc != LAT_OK) return rc;
    apply_choice(lt, pick);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = pick;
    append_tune_file(key, pick);
    return LAT_OK;
}

int sweep_impl(lattice *lt, int64_t n)
{
    if (n < 0) return LAT_EINVAL;
    if (n == 0) return LAT_OK;
    int rc = ensure_series(lt, (unsigned long long)(lt->sweeps + n));
    if (rc != LAT_OK) return rc;
    int64_t left = n;
    if (lt->kernel == LAT_KERNEL_AUTO && lt->tuned_kernel == 0 && lt->P.layout == LAT_INT8 &&
        lt->dynamics == LAT_DYNAMICS_CHECKERBOARD && lt->geom.cpl == nullptr) {
        const int64_t before = lt->sweeps;
        rc = autotune(lt, left);
        if (rc != LAT_OK) return rc;
        n -= lt->sweeps - before;   // sweeps already done (and counted) by the tuner
        if (left == 0) return LAT_OK;
    }
    // The resident kernel runs many sweeps per launch: no graph needed.
    const int gk = (lt->dynamics == LAT_DYNAMICS_CHECKERBOARD && choose_kernel(lt) == LAT_KERNEL_RESIDENT)
                       ? 0 : lt->graph_sweeps;
    if (gk > 0 && left >= gk) {
        rc = ensure_graph(lt);
        if (rc != LAT_OK) return rc;
        while (left >= gk) {
            cudaError_t e = cudaGraphLaunch(lt->graph_exec, lt->stream);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            left -= gk;
        }
    }
    if (left > 0) {
        rc = enqueue_sweeps(lt, left, lt->stream);
        if (rc != LAT_OK) return rc;
    }
    lt->sweeps += n;
    return LAT_OK;
}

static void release(lattice *lt)
{
    if (lt == nullptr) return;
    if (lt->graph_exec) cudaGraphExecDestroy(lt->graph_exec);
    if (lt->cap_stream) cudaStreamDestroy(lt->cap_stream);
    cudaStream_t st = lt->stream;
    dev_free(lt->spins[0], st);
    dev_free(lt->spins[1], st);
    dev_free(lt->bits[0], st);
    dev_free(lt->bits[1], st);
    dev_free(lt->flags, st);
    dev_free(lt->tab, st);
    dev_free(lt->ctrl, st);
    dev_free(lt->series, st);
    dev_free(lt->scratch4, st);
    dev_free(lt->ref, st);
    dev_free(lt->ref_bits, st);
    dev_free(lt->rs_scratch, st);
    dev_free(lt->cpl, st);
    delete lt;
}

int create_impl(lattice_t **out, int dims, int L, int two_S, int model, double J, double h,
                double T_or_c, uint64_t seed, int init, int layout, void *cuda_stream)
{
    if (out == nullptr) return LAT_EINVAL;
    *out = nullptr;
    Params P{};
    int rc = validate(dims, L, two_S, model, J, h, T_or_c, init, layout, P);
    if (rc != LAT_OK) return rc;
    P.seed = seed;
    lattice *lt = new (std::nothrow) lattice();
    if (lt == nullptr) return LAT_ENOMEM;
    lt->P = P;
    lt->stream = (cudaStream_t)cuda_stream;
    cudaStream_t st = lt->stream;

    std::vector<TabEntry> tab;
    int dsmax, nmax, nn;
    build_table(P, tab, dsmax, nmax, nn);
    lt->host_tab = tab;

    Geom &g = lt->geom;
    g.dims = dims;
    g.L = L;
    g.two_S = two_S;
    g.model = model;
    g.cmode = P.cmode;
    g.sh = (two_S == 1) ? 2 : 1;
    g.G = (uint32_t)(((uint32_t)(L / 2) + (1u << g.sh) - 1) >> g.sh);
    g.rows = (uint32_t)(dims == 3 ? (uint64_t)L * L : (uint64_t)L);
    g.N = P.N;
    g.key0 = (uint32_t)(seed & 0xffffffffu);
    g.key1 = (uint32_t)(seed >> 32);
    g.dsmax = dsmax;
    g.nmax = nmax;
    g.nn = nn;
    g.tab_n = (int)tab.size();
    g.bw = (uint32_t)(((uint32_t)(L / 2) + 31) / 32);
    g.half = (uint32_t)(L / 2);
    g.plane = P.N / 2;
    compact_table(g, tab.data());
    // The bit-packed kernel needs whole 32-site words per plane row and a
    // table without never-accept entries.
    if (layout == LAT_BITPACKED) {
        Geom probe = g;
        probe.bits[0] = reinterpret_cast<uint32_t *>(1);
        if (!bitpacked_supported(probe)) {
            delete lt;
            return LAT_ENOTSUP;
        }
    }

    cudaError_t e = dev_alloc((void **)&lt->spins[0], (size_t)P.N, st);
    if (e == cudaSuccess) e = dev_alloc((void **)&lt->spins[1], (size_t)P.N, st);
    if (e == cudaSuccess && model == LAT_NE) e = dev_alloc((void **)&lt->flags, flag_bytes(P), st);
    if (e == cudaSuccess && layout == LAT_BITPACKED) {
        e = dev_alloc((void **)&lt->bits[0], (size_t)2 * L * g.bw * 4, st);
        if (e == cudaSuccess) e = dev_alloc((void **)&lt->bits[1], (size_t)2 * L * g.bw * 4, st);
    }
    if (e == cudaSuccess) e = dev_alloc((void **)&lt->tab, tab.size() * sizeof(TabEntry), st);
    if (e == cudaSuccess) e = dev_alloc((void **)&lt->ctrl, sizeof(Ctrl), st);
    if (e == cudaSuccess) e = dev_alloc((void **)&lt->scratch4, 8 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) {
        rc = (e == cudaErrorMemoryAllocation) ? LAT_ENOMEM : cuda_fail(e, "alloc");
        release(lt);
        return rc;
    }
    g.s[0] = lt->spins[0];
    g.s[1] = lt->spins[1];
    g.bits[0] = lt->bits[0];
    g.bits[1] = lt->bits[1];
    g.flags = lt->flags;
    g.tab = lt->tab;
    g.ctrl = lt->ctrl;

    e = cudaMemcpyAsync(lt->tab, tab.data(), tab.size() * sizeof(TabEntry), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(lt->ctrl, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess && lt->flags) e = cudaMemsetAsync(lt->flags, 0, flag_bytes(P), st);
    if (e == cudaSuccess) e = launch_init(g, init, P.c, st);
    if (e == cudaSuccess && layout == LAT_BITPACKED) e = launch_pack_bits(g, lt->spins[0], lt->bits[0], st);
    // The host table must outlive the async copy: wait once at creation.
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "create");
        release(lt);
        return rc;
    }
    lt->kernel = LAT_KERNEL_AUTO;
    lt->tile_w = 0;
    lt->tile_h = 0;
    lt->graph_sweeps = default_graph_sweeps(P);
    rc = ensure_series(lt, 64);
    if (rc != LAT_OK) {
        release(lt);
        return rc;
    }
    *out = lt;
    return LAT_OK;
}

}  // namespace lat

using namespace lat;

extern "C" {

int lattice_create(lattice_t **out, int dims, int L, int two_S, int model, double J, double h,
                   double T_or_c, uint64_t seed, int init, int layout, void *cuda_stream)
{
    return create_impl(out, dims, L, two_S, model, J, h, T_or_c, seed, init, layout, cuda_stream);
}

int lattice_sweep(lattice_t *lt, int64_t n)
{
    if (lt == nullptr) return LAT_EINVAL;
    return sweep_impl(lt, n);
}

// The planar int8 spins of the current state and a scratch buffer of N
// bytes that is free until the next sweep (the idle half of the double
// buffer; for the bit-packed layout both int8 buffers are staging).
static int current_planar(lattice *lt, int8_t **cur, int8_t **scratch)
{
    const int par = (int)(lt->sweeps & 1);
    if (lt->P.layout == LAT_BITPACKED) {
        cudaError_t e = launch_unpack_bits(lt->geom, lt->bits[par], lt->spins[0], lt->stream);
        if (e != cudaSuccess) return cuda_fail(e, "unpack");
        *cur = lt->spins[0];
        if (scratch) *scratch = lt->spins[1];
    } else {
        *cur = lt->spins[par];
        if (scratch) *scratch = lt->spins[par ^ 1];
    }
    return LAT_OK;
}

// bond, mag, up, unflipped and the field sum of the current state: the
// last recorded sweep's counters, or measured when no sweep is recorded
// (or the couplings or field signs changed after it).
static int current_counters(lattice *lt, long long c[5])
{
    cudaError_t e;
    if (lt->sweeps > lt->series_first && lt->sweeps > lt->disorder_from) {
        const unsigned long long k = (unsigned long long)(lt->sweeps - 1 - lt->series_first);
        e = cudaMemcpyAsync(c, lt->series + 4ull * k, 4 * sizeof(long long), cudaMemcpyDeviceToHost, lt->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c + 4, lt->series + 5 * lt->series_cap + k, sizeof(long long),
                                cudaMemcpyDeviceToHost, lt->stream);
    } else {
        int8_t *cur = nullptr;
        int rc = current_planar(lt, &cur, nullptr);
        if (rc != LAT_OK) return rc;
        e = cudaMemsetAsync(lt->scratch4, 0, 5 * sizeof(long long), lt->stream);
        if (e == cudaSuccess) e = launch_measure(lt->geom, cur, lt->scratch4, lt->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c, lt->scratch4, 5 * sizeof(long long), cudaMemcpyDeviceToHost,
                                lt->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "counters");
    return LAT_OK;
}

int lattice_observables(lattice_t *lt, double *E, double *M, double *density, double *persistence)
{
    if (lt == nullptr) return LAT_EINVAL;
    long long c[5];
    int rc = current_counters(lt, c);
    if (rc != LAT_OK) return rc;
    const double N = (double)lt->P.N;
    double J = lt->P.J, h = lt->P.h;
    if (lt->P.cmode) {
        J = 0.0;
        h = -1.0;
    }
    // Eq. 1: the field term is -h sum_i eta_i s_i (eta = 1 without field signs)
    const double fs = lt->has_fields ? (double)c[4] : (double)c[1];
    if (E) *E = (-J * (double)c[0] - h * fs) / N;
    if (M) *M = (double)c[1] / N;
    if (density) *density = (double)c[2] / N;
    if (persistence) *persistence = (lt->P.model == LAT_NE) ? (double)c[3] / N : NAN;
    return LAT_OK;
}

int lattice_series(lattice_t *lt, int64_t first, int64_t count, int64_t *bond, int64_t *mag,
                   int64_t *up, int64_t *unflipped)
{
    if (lt == nullptr || first < 0 || count < 0) return LAT_EINVAL;
    if (first < lt->series_first || first + count > lt->sweeps) return LAT_ERANGE;
    if (count == 0) return LAT_OK;
    std::vector<long long> buf((size_t)count * 4);
    cudaError_t e = cudaMemcpyAsync(buf.data(),
                                    lt->series + 4ull * (unsigned long long)(first - lt->series_first),
                                    (size_t)count * 4 * sizeof(long long), cudaMemcpyDeviceToHost,
                                    lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "series copy");
    for (int64_t k = 0; k < count; ++k) {
        if (bond) bond[k] = buf[4 * k + 0];
        if (mag) mag[k] = buf[4 * k + 1];
        if (up) up[k] = buf[4 * k + 2];
        if (unflipped) unflipped[k] = buf[4 * k + 3];
    }
    return LAT_OK;
}

int lattice_set_reference(lattice_t *lt, int64_t *ref_sweep)
{
    if (lt == nullptr) return LAT_EINVAL;
    cudaStream_t st = lt->stream;
    cudaError_t e = cudaSuccess;
    if (lt->P.layout == LAT_BITPACKED) {
        if (lt->ref_bits == nullptr) e = dev_alloc((void **)&lt->ref_bits, bits_bytes(lt->P), st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lt->ref_bits, lt->bits[lt->sweeps & 1], bits_bytes(lt->P), cudaMemcpyDeviceToDevice,
                                st);
        lt->geom.ref_bits = lt->ref_bits;
    } else {
        if (lt->ref == nullptr) e = dev_alloc((void **)&lt->ref, (size_t)lt->P.N, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lt->ref, lt->spins[lt->sweeps & 1], (size_t)lt->P.N, cudaMemcpyDeviceToDevice, st);
        lt->geom.ref = lt->ref;
    }
    if (e != cudaSuccess) {
        lt->geom.ref = nullptr;
        lt->geom.ref_bits = nullptr;
        lt->ref_sweep = -1;
        return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "set reference");
    }
    lt->ref_sweep = lt->sweeps;
    lt->graph_valid = false;   // the descriptor captured in a graph changed
    if (ref_sweep) *ref_sweep = lt->ref_sweep;
    return LAT_OK;
}

int lattice_set_dynamics(lattice_t *lt, int dynamics, int tile, int lambda)
{
    if (lt == nullptr) return LAT_EINVAL;
    if (dynamics == LAT_DYNAMICS_CHECKERBOARD) {
        lt->dynamics = dynamics;
        lt->graph_valid = false;
        return LAT_OK;
    }
    if (dynamics != LAT_DYNAMICS_RANDOM_SITE && dynamics != LAT_DYNAMICS_RANDOM_SITE_BALANCED) return LAT_EINVAL;
    if (lt->P.dims != 2 || lt->P.two_S != 1 || lt->P.layout != LAT_INT8 || lt->cpl != nullptr ||
        lt->P.model == LAT_POTTS)
        return LAT_ENOTSUP;
    if (!rsite_params_ok(lt->geom, tile, lambda, dynamics == LAT_DYNAMICS_RANDOM_SITE_BALANCED)) return LAT_EINVAL;
    if (lt->rs_scratch == nullptr) {
        cudaError_t e = dev_alloc((void **)&lt->rs_scratch, (size_t)lt->P.N, lt->stream);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "random-site scratch");
    }
    lt->dynamics = dynamics;
    lt->rs_tile = tile;
    lt->rs_lambda = lambda;
    lt->graph_valid = false;
    return LAT_OK;
}

// Upload the host disorder bytes (or drop the device copy when every byte
// is zero) and rebuild the acceptance table: a second half for -h follows
// the first while field signs are set.
static int apply_disorder(lattice *lt)
{
    cudaStream_t st = lt->stream;
    cudaError_t e = cudaStreamSynchronize(st);   // no queued sweep may read the old table or bytes
    if (e != cudaSuccess) return cuda_fail(e, "disorder sync");
    std::vector<TabEntry> tab;
    int dsmax, nmax, nn;
    build_table(lt->P, tab, dsmax, nmax, nn);
    lt->fields_wide_ok = false;
    if (lt->has_fields) {
        Params Pm = lt->P;
        Pm.h = -Pm.h;
        std::vector<TabEntry> neg;
        build_table(Pm, neg, dsmax, nmax, nn);
        // the 2D wide kernel takes the -h entries in t' = thr - 1 form: no
        // never-accept entry among the reachable ones
        Geom probe = lt->geom;
        compact_table(probe, neg.data());
        lt->fields_wide_ok = true;
        for (int k = 0; k < 16; ++k)
            if ((k & 7) <= 4 && !((probe.always16 >> k) & 1u) && probe.thr16[k] == 0u) lt->fields_wide_ok = false;
        tab.insert(tab.end(), neg.begin(), neg.end());
    }
    if ((int)tab.size() != lt->geom.tab_n) {
        TabEntry *t = nullptr;
        e = dev_alloc((void **)&t, tab.size() * sizeof(TabEntry), st);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "table alloc");
        dev_free(lt->tab, st);
        lt->tab = t;
        lt->geom.tab = t;
        lt->geom.tab_n = (int)tab.size();
    }
    e = cudaMemcpyAsync(lt->tab, tab.data(), tab.size() * sizeof(TabEntry), cudaMemcpyHostToDevice, st);
    const bool any = lt->has_bonds || lt->has_fields;
    if (e == cudaSuccess && any) {
        if (lt->cpl == nullptr) e = dev_alloc((void **)&lt->cpl, (size_t)lt->P.N, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lt->cpl, lt->dis_host.data(), (size_t)lt->P.N, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host vectors go out of scope
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "set disorder");
    if (!any) {
        dev_free(lt->cpl, st);
        lt->cpl = nullptr;
        lt->dis_host.clear();
    }
    lt->geom.cpl = lt->cpl;
    lt->disorder_from = lt->sweeps;
    lt->graph_valid = false;
    return LAT_OK;
}

// Checks shared by the coupling and field setters: Ising, int8 layout,
// checkerboard dynamics.
static int disorder_ok(const lattice *lt)
{
    const Params &P = lt->P;
    if (P.model != LAT_ISING || P.layout != LAT_INT8 || lt->dynamics != LAT_DYNAMICS_CHECKERBOARD)
        return LAT_ENOTSUP;
    return LAT_OK;
}

int lattice_set_couplings(lattice_t *lt, const int8_t *bond_signs)
{
    if (lt == nullptr) return LAT_EINVAL;
    const Params &P = lt->P;
    const uint64_t N = P.N;
    if (bond_signs == nullptr) {
        if (!lt->has_bonds) return LAT_OK;
        for (auto &b : lt->dis_host) b &= 0x40u;   // keep the field signs
        lt->has_bonds = false;
        return apply_disorder(lt);
    }
    int rc = disorder_ok(lt);
    if (rc != LAT_OK) return rc;
    for (uint64_t i = 0; i < (uint64_t)P.dims * N; ++i)
        if (bond_signs[i] != 1 && bond_signs[i] != -1) return LAT_EINVAL;
    // One byte per site (planar layout): bit 2d = bond to -e_d negative,
    // bit 2d+1 = bond to +e_d negative; the -e_d bond is the +e_d bond of
    // the neighbour behind.
    const int L = P.L;
    if (lt->dis_host.size() != (size_t)N) lt->dis_host.assign((size_t)N, 0u);
    for (uint64_t i = 0; i < N; ++i) {
        const int x = (int)(i % (uint64_t)L), y = (int)((i / (uint64_t)L) % (uint64_t)L);
        const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
        const int c[3] = {x, y, z};
        uint32_t b = 0;
        for (int d = 0; d < P.dims; ++d) {
            int nb[3] = {x, y, z};
            nb[d] = (c[d] + L - 1) % L;
            const uint64_t back = (uint64_t)nb[0] + (uint64_t)L * ((uint64_t)nb[1] + (uint64_t)L * (uint64_t)nb[2]);
            if (bond_signs[(uint64_t)d * N + back] < 0) b |= 1u << (2 * d);
            if (bond_signs[(uint64_t)d * N + i] < 0) b |= 1u << (2 * d + 1);
        }
        uint8_t &dst = lt->dis_host[planar_index(lt->geom, x, y, z)];
        dst = (uint8_t)((dst & 0x40u) | b);
    }
    lt->has_bonds = true;
    return apply_disorder(lt);
}

int lattice_set_fields(lattice_t *lt, const int8_t *field_signs)
{
    if (lt == nullptr) return LAT_EINVAL;
    const Params &P = lt->P;
    const uint64_t N = P.N;
    if (field_signs == nullptr) {
        if (!lt->has_fields) return LAT_OK;
        for (auto &b : lt->dis_host) b &= 0x3fu;   // keep the coupling signs
        lt->has_fields = false;
        return apply_disorder(lt);
    }
    int rc = disorder_ok(lt);
    if (rc != LAT_OK) return rc;
    for (uint64_t i = 0; i < N; ++i)
        if (field_signs[i] != 1 && field_signs[i] != -1) return LAT_EINVAL;
    const int L = P.L;
    if (lt->dis_host.size() != (size_t)N) lt->dis_host.assign((size_t)N, 0u);
    for (uint64_t i = 0; i < N; ++i) {
        const int x = (int)(i % (uint64_t)L), y = (int)((i / (uint64_t)L) % (uint64_t)L);
        const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
        uint8_t &dst = lt->dis_host[planar_index(lt->geom, x, y, z)];
        dst = (uint8_t)((dst & 0x3fu) | (field_signs[i] < 0 ? 0x40u : 0u));
    }
    lt->has_fields = true;
    rc = apply_disorder(lt);
    if (rc == LAT_OK) lt->fields_from = lt->sweeps;
    return rc;
}

int lattice_field_series(lattice_t *lt, int64_t first, int64_t count, int64_t *field)
{
    if (lt == nullptr || first < 0 || count < 0) return LAT_EINVAL;
    if (!lt->has_fields) return LAT_ENOENT;
    if (first < lt->series_first || first < lt->fields_from || first + count > lt->sweeps) return LAT_ERANGE;
    if (count == 0 || field == nullptr) return LAT_OK;
    cudaError_t e = cudaMemcpyAsync(field,
                                    lt->series + 5 * lt->series_cap + (unsigned long long)(first - lt->series_first),
                                    (size_t)count * sizeof(int64_t), cudaMemcpyDeviceToHost, lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "field series copy");
    return LAT_OK;
}

int lattice_clear_reference(lattice_t *lt)
{
    if (lt == nullptr) return LAT_EINVAL;
    dev_free(lt->ref, lt->stream);
    dev_free(lt->ref_bits, lt->stream);
    lt->ref = nullptr;
    lt->ref_bits = nullptr;
    lt->geom.ref = nullptr;
    lt->geom.ref_bits = nullptr;
    lt->ref_sweep = -1;
    lt->graph_valid = false;
    return LAT_OK;
}

int lattice_autocorrelation(lattice_t *lt, int64_t first, int64_t count, double m, int64_t *overlap,
                            double *phi)
{
    if (lt == nullptr || first < 0 || count < 0) return LAT_EINVAL;
    if (lt->ref_sweep < 0) return LAT_ENOENT;
    if (std::isnan(m)) {
        // the model's own polarisation: m = <s_i> = 2c - 1 for the North-East
        // model at concentration c (§III.B, Eq. 4); other lattices have none
        if (lt->P.model == LAT_NE && lt->P.cmode) m = 2.0 * lt->P.c - 1.0;
        else if (phi != nullptr) return LAT_EINVAL;
    }
    if (phi != nullptr && !(std::fabs(m) < 1.0)) return LAT_EINVAL;
    if (first < lt->series_first || first < lt->ref_sweep || first + count > lt->sweeps) return LAT_ERANGE;
    if (count == 0) return LAT_OK;
    std::vector<long long> buf((size_t)count);
    cudaError_t e = cudaMemcpyAsync(buf.data(),
                                    lt->series + 4 * lt->series_cap + (unsigned long long)(first - lt->series_first),
                                    (size_t)count * sizeof(long long), cudaMemcpyDeviceToHost, lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "autocorrelation copy");
    const double N = (double)lt->P.N, m2 = m * m;
    for (int64_t k = 0; k < count; ++k) {
        if (overlap) overlap[k] = buf[(size_t)k];
        if (phi) phi[k] = ((double)buf[(size_t)k] / N - m2) / (1.0 - m2);
    }
    return LAT_OK;
}

int lattice_get_spins(lattice_t *lt, int8_t *host_out)
{
    if (lt == nullptr || host_out == nullptr) return LAT_EINVAL;
    int8_t *cur = nullptr, *lin = nullptr;
    int rc = current_planar(lt, &cur, &lin);
    if (rc != LAT_OK) return rc;
    cudaError_t e = launch_to_linear(lt->geom, cur, lin, lt->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, lin, (size_t)lt->P.N, cudaMemcpyDeviceToHost, lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get spins");
    return LAT_OK;
}

static bool spins_allowed(const Params &P, const int8_t *s)
{
    // Branch-free scan (vectorises): count values outside the allowed set.
    if (P.model == LAT_POTTS) {
        uint64_t bad = 0;
        for (uint64_t i = 0; i < P.N; ++i) bad += (uint64_t)((s[i] < 0) | (s[i] > P.two_S));
        return bad == 0;
    }
    const int smax = max_spin(P.two_S);
    const int odd = P.two_S & 1;
    uint64_t bad = 0;
    for (uint64_t i = 0; i < P.N; ++i) {
        const int v = s[i];
        bad += (uint64_t)((v < -smax) | (v > smax) | (odd & ((v + P.two_S) & 1)));
    }
    return bad == 0;
}

// Copy host spins (x fastest) into the current-state buffer: upload to the
// idle buffer, convert to planar (and pack for the bit-packed layout).
static cudaError_t put_spins(lattice *lt, const int8_t *host_in)
{
    const int par = (int)(lt->sweeps & 1);
    int8_t *lin = (lt->P.layout == LAT_BITPACKED) ? lt->spins[1] : lt->spins[par ^ 1];
    int8_t *dst = (lt->P.layout == LAT_BITPACKED) ? lt->spins[0] : lt->spins[par];
    cudaError_t e = cudaMemcpyAsync(lin, host_in, (size_t)lt->P.N, cudaMemcpyHostToDevice, lt->stream);
    if (e == cudaSuccess) e = launch_to_planar(lt->geom, lin, dst, lt->stream);
    if (e == cudaSuccess && lt->P.layout == LAT_BITPACKED)
        e = launch_pack_bits(lt->geom, dst, lt->bits[par], lt->stream);
    return e;
}

// Persistence flags: device bytes (one per Philox group of each colour
// plane row, bit q = site 4m+q) <-> one host byte per site, x fastest.
static void flags_to_host(const lattice *lt, const std::vector<uint8_t> &dev, uint8_t *out)
{
    const Geom &g = lt->geom;
    const int L = g.L;
    for (uint64_t i = 0; i < g.N; ++i) {
        const int x = (int)(i % (uint64_t)L);
        const int y = (int)((i / (uint64_t)L) % (uint64_t)L);
        const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
        const int c = (x + y + z) & 1;
        const uint64_t r = (uint64_t)y + (uint64_t)L * (uint64_t)z;
        const uint32_t j = (uint32_t)x >> 1;
        const uint8_t f = dev[((uint64_t)c * g.rows + r) * g.G + (j >> g.sh)];
        out[i] = (uint8_t)((f >> (j & ((1u << g.sh) - 1u))) & 1u);
    }
}

static void flags_from_host(const lattice *lt, const uint8_t *in, std::vector<uint8_t> &dev)
{
    const Geom &g = lt->geom;
    const int L = g.L;
    for (uint64_t i = 0; i < g.N; ++i) {
        if (!in[i]) continue;
        const int x = (int)(i % (uint64_t)L);
        const int y = (int)((i / (uint64_t)L) % (uint64_t)L);
        const int z = (int)(i / ((uint64_t)L * (uint64_t)L));
        const int c = (x + y + z) & 1;
        const uint64_t r = (uint64_t)y + (uint64_t)L * (uint64_t)z;
        const uint32_t j = (uint32_t)x >> 1;
        dev[((uint64_t)c * g.rows + r) * g.G + (j >> g.sh)] |= (uint8_t)(1u << (j & ((1u << g.sh) - 1u)));
    }
}

int lattice_set_spins(lattice_t *lt, const int8_t *host_in)
{
    if (lt == nullptr || host_in == nullptr) return LAT_EINVAL;
    // Upload into the idle buffer and check the values there (on the device,
    // not by a host scan of N bytes); only then convert into the current
    // buffer, so a rejected array leaves the lattice unchanged.
    const int par = (int)(lt->sweeps & 1);
    int8_t *lin = (lt->P.layout == LAT_BITPACKED) ? lt->spins[1] : lt->spins[par ^ 1];
    int8_t *dst = (lt->P.layout == LAT_BITPACKED) ? lt->spins[0] : lt->spins[par];
    unsigned long long bad = 0;
    cudaError_t e = cudaMemcpyAsync(lin, host_in, (size_t)lt->P.N, cudaMemcpyHostToDevice, lt->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lt->scratch4, 0, sizeof(unsigned long long), lt->stream);
    if (e == cudaSuccess) e = launch_count_bad(lt->geom, lin, lt->scratch4, lt->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, lt->scratch4, sizeof bad, cudaMemcpyDeviceToHost, lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);   // the caller may reuse host_in now
    if (e != cudaSuccess) return cuda_fail(e, "set spins");
    if (bad != 0) return LAT_EINVAL;
    e = launch_to_planar(lt->geom, lin, dst, lt->stream);
    if (e == cudaSuccess && lt->P.layout == LAT_BITPACKED) e = launch_pack_bits(lt->geom, dst, lt->bits[par], lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set spins");
    return LAT_OK;
}

int lattice_get_state(lattice_t *lt, int8_t *spins, uint8_t *flags, int64_t *sweeps)
{
    if (lt == nullptr) return LAT_EINVAL;
    if (spins) {
        int rc = lattice_get_spins(lt, spins);
        if (rc != LAT_OK) return rc;
    }
    if (flags) {
        if (lt->flags) {
            std::vector<uint8_t> dev(flag_bytes(lt->P));
            cudaError_t e = cudaMemcpyAsync(dev.data(), lt->flags, dev.size(), cudaMemcpyDeviceToHost,
                                            lt->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
            if (e != cudaSuccess) return cuda_fail(e, "get flags");
            flags_to_host(lt, dev, flags);
        } else {
            memset(flags, 0, (size_t)lt->P.N);
        }
    }
    if (sweeps) *sweeps = lt->sweeps;
    return LAT_OK;
}

int lattice_set_state(lattice_t *lt, const int8_t *spins, const uint8_t *flags, int64_t sweeps)
{
    if (lt == nullptr || spins == nullptr || sweeps < 0) return LAT_EINVAL;
    if (!spins_allowed(lt->P, spins)) return LAT_EINVAL;
    std::vector<uint8_t> dev;
    if (lt->flags) {
        dev.assign(flag_bytes(lt->P), 0u);
        if (flags) flags_from_host(lt, flags, dev);
    }
    cudaError_t e = cudaStreamSynchronize(lt->stream);
    const int64_t old_sweeps = lt->sweeps;
    lt->sweeps = sweeps;  // selects the buffer parity put_spins writes
    if (e == cudaSuccess) e = put_spins(lt, spins);
    if (e == cudaSuccess && lt->flags)
        e = cudaMemcpyAsync(lt->flags, dev.data(), dev.size(), cudaMemcpyHostToDevice, lt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) {
        lt->sweeps = old_sweeps;
        return cuda_fail(e, "set state");
    }
    // The recorded series restarts at the restored sweep index.
    dev_free(lt->series, lt->stream);
    lt->series = nullptr;
    lt->series_cap = 0;
    lt->sweeps = sweeps;
    lt->series_first = sweeps;
    lt->disorder_from = sweeps;
    lt->fields_from = sweeps;
    return ensure_series(lt, (unsigned long long)sweeps + 64);
}

int lattice_info(lattice_t *lt, int64_t *sweeps, int64_t *n_sites, int64_t *device_bytes)
{
    if (lt == nullptr) return LAT_EINVAL;
    if (sweeps) *sweeps = lt->sweeps;
    if (n_sites) *n_sites = (int64_t)lt->P.N;
    if (device_bytes)
        *device_bytes = (int64_t)(footprint_bytes(lt->P) +
                                  (size_t)lt->series_cap * 6 * sizeof(long long) +
                                  (lt->ref ? (size_t)lt->P.N : 0) +
                                  (lt->ref_bits ? bits_bytes(lt->P) : 0) +
                                  (lt->rs_scratch ? (size_t)lt->P.N : 0));
    return LAT_OK;
}

int lattice_device_spins(lattice_t *lt, void **dev_ptr, size_t *bytes)
{
    if (lt == nullptr || dev_ptr == nullptr) return LAT_EINVAL;
    const int par = (int)(lt->sweeps & 1);
    if (lt->P.layout == LAT_BITPACKED) {
        *dev_ptr = lt->bits[par];
        if (bytes) *bytes = (size_t)2 * lt->P.L * lt->geom.bw * 4;
    } else {
        *dev_ptr = lt->spins[par];
        if (bytes) *bytes = (size_t)lt->P.N;
    }
    return LAT_OK;
}

int lattice_set_kernel(lattice_t *lt, int kernel, int tile_w, int tile_h, int sweeps_per_graph)
{
    if (lt == nullptr) return LAT_EINVAL;
    if (kernel < LAT_KERNEL_AUTO || kernel > LAT_KERNEL_RESIDENT) return LAT_EINVAL;
    if (tile_w < 0 || tile_h < 0 || sweeps_per_graph < 0) return LAT_EINVAL;
    if (kernel == LAT_KERNEL_TILED && !tiled_supported(lt->geom)) return LAT_ENOTSUP;
    if (kernel == LAT_KERNEL_WIDE &&
        (!any_wide(lt->geom) || (lt->has_fields && !(wide_supported(lt->geom) && lt->fields_wide_ok))))
        return LAT_ENOTSUP;
    if (kernel == LAT_KERNEL_RESIDENT && !resident_supported(lt->geom)) return LAT_ENOTSUP;
    if (!tile_shape_ok(tile_w, tile_h)) return LAT_EINVAL;
    lt->kernel = kernel;
    lt->tile_w = tile_w;
    lt->tile_h = tile_h;
    lt->graph_sweeps = sweeps_per_graph ? sweeps_per_graph : default_graph_sweeps(lt->P);
    lt->graph_pinned = sweeps_per_graph != 0;
    lt->graph_valid = false;
    return LAT_OK;
}

int lattice_get_kernel(lattice_t *lt, int *kernel, int *tile_w, int *tile_h, int *sweeps_per_graph)
{
    if (lt == nullptr) return LAT_EINVAL;
    const int k = choose_kernel(lt);
    if (kernel) *kernel = (k == LAT_KERNEL_AUTO) ? LAT_KERNEL_GENERIC : k;
    if (tile_w) *tile_w = (k == LAT_KERNEL_TILED) ? 256 : 0;
    if (tile_h) *tile_h = (k == LAT_KERNEL_TILED) ? (lt->tile_h ? lt->tile_h : default_tile_h()) : 0;
    if (sweeps_per_graph) *sweeps_per_graph = lt->graph_sweeps;
    return LAT_OK;
}

int lattice_threshold_table(int dims, int two_S, int model, double J, double h, double T_or_c,
                            uint32_t *thr, uint8_t *always, int cap, int *count, int *dsmax,
                            int *nmax)
{
    Params P{};
    const int init = (model == LAT_NE && J == 0.0 && h == 0.0) ? LAT_INIT_EQUILIBRIUM : LAT_INIT_COLD;
    int rc = validate(dims, 2, two_S, model, J, h, T_or_c, init, LAT_INT8, P);
    if (rc != LAT_OK) return rc;
    std::vector<TabEntry> tab;
    int dm, nm, nn;
    build_table(P, tab, dm, nm, nn);
    const int n = (int)tab.size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (thr) thr[i] = tab[i].thr;
        if (always) always[i] = (uint8_t)tab[i].always;
    }
    if (count) *count = n;
    if (dsmax) *dsmax = dm;
    if (nmax) *nmax = nm;
    return LAT_OK;
}

int lattice_synchronize(lattice_t *lt)
{
    if (lt == nullptr) return LAT_EINVAL;
    cudaError_t e = cudaStreamSynchronize(lt->stream);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return LAT_OK;
}

void lattice_destroy(lattice_t *lt) { release(lt); }

const char *lattice_strerror(int code)
{
    switch (code) {
    case LAT_OK: return "success";
    case LAT_EINVAL: return "invalid argument";
    case LAT_ENOMEM: return "out of memory";
    case LAT_ECUDA: return "CUDA error";
    case LAT_ETIMEOUT: return "device-side wait timed out";
    case LAT_EBUSY: return "not ready";
    case LAT_ENOTSUP: return "not supported";
    case LAT_ERANGE: return "out of range";
    case LAT_ENOENT: return "no such id";
    default: return "unknown error";
    }
}

const char *lattice_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

const char *lattice_version(void) { return "lattice-gb300 1.0 (sm_103a)"; }

// Test hook (not part of the documented API surface): the countdown-th next
// device allocation fails with out-of-memory.
int lattice_test_fail_alloc(int countdown)
{
    g_fail_alloc_countdown.store(countdown < 0 ? 0 : countdown);
    return LAT_OK;
}

}  // extern "C"
