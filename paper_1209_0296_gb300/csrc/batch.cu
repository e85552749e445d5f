// batch.cu -- the batched engine behind lattice_batch_*: many lattices of
// any sizes and models advanced together.  Each sweep step is a set of
// persistent-grid launches over work lists: two (colour 0, colour 1) per
// model over (lattice, item) pairs of the 2D spin-1/2 wide kernel, one over
// (lattice, tile) items of lattices set to the fused tiled kernel, two over
// (lattice, item) pairs of the 3D / spin-S wide kernel and two over
// (lattice, chunk) pairs of the generic kernel; then one small kernel
// advances every lattice's sweep counter.  Small 2D spin-1/2 lattices
// instead run as resident CTAs (one CTA per lattice holding it in shared
// memory for all its sweeps) on a side stream, concurrently with the step
// loop of the others.  Steps with the same set of lattices are captured
// once in a CUDA graph and replayed.  Every lattice keeps its own seed,
// table and sweep counter, so its result is bit-identical to running it
// alone.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "lattice_capi_internal.h"

using namespace lat;

// Device arrays of one run (descriptors, work items, control pointers, the
// resident lattices' descriptors and sweep counts) with their pinned host
// staging.  Runs take the slots in turn and a slot is reused only after the
// run that last used it has finished (its event), so a run's uploads never
// wait for the work queued before it: the host can queue run k+1 while run k
// executes.
struct BatchSlot {
    Geom *d_geoms = nullptr;
    int geoms_cap = 0;
    uint2 *d_items = nullptr;  // tiled items, then wide items, then Potts items, then generic items
    int items_cap = 0;
    Ctrl **d_ctrls = nullptr;
    int ctrls_cap = 0;
    Geom *d_res_geoms = nullptr;
    int res_geoms_cap = 0;
    long long *d_res_n = nullptr;
    int res_n_cap = 0;
    char *h_pin = nullptr;     // pinned staging of the uploads
    size_t h_cap = 0;
    cudaEvent_t done = nullptr;
    bool used = false;
};
constexpr int kBatchSlots = 3;

struct lattice_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<std::pair<lattice *, int64_t>> pending;
    BatchSlot slots[kBatchSlots];
    int next_slot = 0;
    // The caller orders every other use of the lattices against this batch's
    // stream itself (the server): no per-lattice stream synchronisation
    // before a run and no per-lattice stream waits after it.
    bool caller_orders = false;
    // Recorded on the batch stream right before a run's first device work
    // (after its host preparation), when set: the server's busy-time clock.
    cudaEvent_t start_event = nullptr;
    // The rows per any-L item and steps per graph of the last run (0 rows:
    // the size-based default), as tuned or defaulted.
    int last_passes = 0, last_gsteps = 0;
    // next item of: Ising tiles, NE tiles, generic colour 0 / 1, 3D/spin-S
    // per site colour 0 / 1, 2D Ising wide colour 0 / 1, 2D North-East wide
    // colour 0 / 1, Potts colour 0 / 1, any-L 2D Ising colour 0 / 1, any-L 2D
    // North-East colour 0 / 1, 3D/spin-S byte-parallel colour 0 / 1, 2D
    // c-mode North-East wide colour 0 / 1, any-L 2D c-mode North-East
    // colour 0 / 1
    unsigned *d_counters = nullptr;
    int grid_tiled_ising = 0, grid_tiled_ne = 0, grid_generic = 0, grid_wide[2] = {0, 0}, grid_potts = 0;
    int grid_any[2] = {0, 0};     // 2D any-L, Ising / North-East
    // resident lattices
    cudaStream_t res_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_done = nullptr;   // end of a run: each lattice's stream waits on it
    std::vector<cudaEvent_t> ev_streams;   // one per distinct lattice stream of a run
};

namespace {

constexpr int kChunk = 256;       // Philox groups per generic item (one CTA)
constexpr int kGraphSteps = 32;   // steps per captured graph
constexpr int kGraphMinSteps = 128;
constexpr int kCounters = 22;
constexpr int kResidentMaxL = 128;      // AUTO lattices up to this size run resident
constexpr int kResidentChunk = 1 << 16; // sweeps per resident launch

template <typename T>
int grow(T **p, int &cap, int need, cudaStream_t st)
{
    if (need <= cap) return LAT_OK;
    int c = cap ? cap : 64;
    while (c < need) c *= 2;
    void *q = nullptr;
    cudaError_t e = dev_alloc(&q, (size_t)c * sizeof(T), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "batch alloc");
    dev_free(*p, st);
    *p = (T *)q;
    cap = c;
    return LAT_OK;
}

// Copy n elements of host data into the slot's pinned staging at byte
// offset `at` (rounded up to 16) and queue their upload to dst; returns the
// next free offset.
template <typename T>
size_t stage(BatchSlot &sl, size_t at, T *dst, const T *src, size_t n, cudaStream_t st, cudaError_t &e)
{
    at = (at + 15) & ~(size_t)15;
    if (e != cudaSuccess || n == 0) return at;
    memcpy(sl.h_pin + at, src, n * sizeof(T));
    e = cudaMemcpyAsync(dst, sl.h_pin + at, n * sizeof(T), cudaMemcpyHostToDevice, st);
    return at + n * sizeof(T);
}

int ensure_pinned(BatchSlot &sl, size_t bytes)
{
    if (bytes <= sl.h_cap) return LAT_OK;
    size_t c = sl.h_cap ? sl.h_cap : 64 * 1024;
    while (c < bytes) c *= 2;
    void *p = nullptr;
    cudaError_t e = cudaMallocHost(&p, c);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "batch staging");
    if (sl.h_pin) cudaFreeHost(sl.h_pin);   // the slot's last run has finished
    sl.h_pin = (char *)p;
    sl.h_cap = c;
    return LAT_OK;
}

// Take the next slot, once the run that used it last has finished.
int take_slot(lattice_batch *b, BatchSlot **out)
{
    BatchSlot &sl = b->slots[b->next_slot];
    b->next_slot = (b->next_slot + 1) % kBatchSlots;
    cudaError_t e = cudaSuccess;
    if (sl.done == nullptr) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    else if (sl.used) e = cudaEventSynchronize(sl.done);
    if (e != cudaSuccess) return cuda_fail(e, "batch slot");
    sl.used = false;
    *out = &sl;
    return LAT_OK;
}

// Item counts of the current active set, in this order in d_items: tiles
// of Ising lattices, tiles of North-East lattices, 2D wide items of Ising
// and of North-East lattices, any-L 2D items of Ising and of North-East
// lattices, 3D / spin-S wide items, Potts items, generic chunks.
struct Shape {
    // n_w2 / n_grp: Ising, North-East at temperature T, North-East in c-mode
    int n_lat, n_ising, n_ne, n_w2[3], n_grp[3], n_wide[2], n_potts, n_gen;
    int passes3, passes_p;   // rows a thread visits per 3D / spin-S item and per Potts item
    int tab_gen;   // largest table among the generic lattices
};

// One phase of a run: its item counts and where its descriptors, items and
// control pointers start in the batch's device arrays.
struct Phase {
    Shape sh;
    int64_t steps;
    const Geom *geoms;
    const uint2 *items;
    Ctrl *const *ctrls;
    int passes;   // rows a thread visits per any-L item (0: the size-based default)
    int gsteps;   // steps per captured graph
};

// The batch tuner's choice for one composition of lattices: rows per
// any-L item and steps per captured graph.
struct BatchTune {
    int passes, gsteps;
};

// Queue `steps` sweep steps of one phase.
int enqueue_steps(lattice_batch *b, const Phase &ph, int steps, cudaStream_t st)
{
    const Shape &sh = ph.sh;
    for (int s = 0; s < steps; ++s) {
        cudaError_t e = cudaSuccess;
        if (sh.n_ising > 0)
            e = launch_batch_tiled(ph.geoms, ph.items, sh.n_ising, b->d_counters + 0, 0, 0,
                                   std::min(b->grid_tiled_ising, sh.n_ising), false, st);
        if (e == cudaSuccess && sh.n_ne > 0)
            e = launch_batch_tiled(ph.geoms, ph.items + sh.n_ising, sh.n_ne, b->d_counters + 1, 0, 0,
                                   std::min(b->grid_tiled_ne, sh.n_ne), true, st);
        const uint2 *w2 = ph.items + sh.n_ising + sh.n_ne;
        // Ising, North-East at T, North-East in c-mode: colour 0, then colour 1
        static const int kCtrW2[3] = {6, 8, 18}, kCtrGrp[3] = {12, 14, 20};
        for (int m = 0; m < 3; ++m) {   // L % 32 == 0
            for (int colour = 0; colour < 2 && e == cudaSuccess && sh.n_w2[m] > 0; ++colour)
                e = launch_batch_any(ph.geoms, w2, sh.n_w2[m], b->d_counters + kCtrW2[m] + colour, colour, m >= 1,
                                     m == 2, true, ph.passes, std::min(b->grid_any[m ? 1 : 0], sh.n_w2[m]), st);
            w2 += sh.n_w2[m];
        }
        for (int m = 0; m < 3; ++m) {   // other even L
            for (int colour = 0; colour < 2 && e == cudaSuccess && sh.n_grp[m] > 0; ++colour)
                e = launch_batch_any(ph.geoms, w2, sh.n_grp[m], b->d_counters + kCtrGrp[m] + colour, colour, m >= 1,
                                     m == 2, false, ph.passes, std::min(b->grid_any[m ? 1 : 0], sh.n_grp[m]), st);
            w2 += sh.n_grp[m];
        }
        const uint2 *wide = w2;
        for (int m = 0; m < 2; ++m) {   // 3D / spin-S: per site, then byte-parallel
            static const int kCtr[2] = {4, 16};
            for (int colour = 0; colour < 2 && e == cudaSuccess && sh.n_wide[m] > 0; ++colour)
                e = launch_batch_wide3(ph.geoms, wide, sh.n_wide[m], b->d_counters + kCtr[m] + colour, colour,
                                       m == 1, sh.passes3, std::min(b->grid_wide[m], sh.n_wide[m]), st);
            wide += sh.n_wide[m];
        }
        const uint2 *potts = wide;
        for (int colour = 0; colour < 2 && e == cudaSuccess && sh.n_potts > 0; ++colour)
            e = launch_batch_potts(ph.geoms, potts, sh.n_potts, b->d_counters + 10 + colour, colour, sh.passes_p,
                                   std::min(b->grid_potts, sh.n_potts), st);
        const uint2 *gen = potts + sh.n_potts;
        if (e == cudaSuccess && sh.n_gen > 0)
            e = launch_batch_generic(ph.geoms, gen, sh.n_gen, b->d_counters + 2, 0, 0,
                                     std::min(b->grid_generic, sh.n_gen), sh.tab_gen, st);
        if (e == cudaSuccess && sh.n_gen > 0)
            e = launch_batch_generic(ph.geoms, gen, sh.n_gen, b->d_counters + 3, 1, 0,
                                     std::min(b->grid_generic, sh.n_gen), sh.tab_gen, st);
        if (e == cudaSuccess) e = launch_batch_advance(ph.ctrls, sh.n_lat, b->d_counters, kCounters, 1ull, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    }
    return LAT_OK;
}

// Capture `steps` steps of a phase in a CUDA graph on the capture stream.
int capture_steps(lattice_batch *b, const Phase &ph, int steps, cudaGraphExec_t *exec)
{
    if (b->cap_stream == nullptr) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "batch capture stream");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "batch begin capture");
    int rc = enqueue_steps(b, ph, steps, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc != LAT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph");
    return LAT_OK;
}

int run_steps(lattice_batch *b, const Phase &ph)
{
    int64_t left = ph.steps;
    // A graph pays for its capture and instantiation (milliseconds) only
    // over many replays; short runs (a serving round) launch directly,
    // which the host enqueues faster than the device drains them.
    if (left >= std::max<int64_t>(kGraphMinSteps, ph.gsteps)) {
        cudaGraphExec_t exec = nullptr;
        int rc = capture_steps(b, ph, ph.gsteps, &exec);
        if (rc != LAT_OK) return rc;
        cudaError_t e = cudaSuccess;
        while (left >= ph.gsteps && e == cudaSuccess) {
            e = cudaGraphLaunch(exec, b->stream);
            left -= ph.gsteps;
        }
        cudaGraphExecDestroy(exec);  // safe: destruction waits for no launch; launches stay valid
        if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    }
    if (left > 0) return enqueue_steps(b, ph, (int)left, b->stream);
    return LAT_OK;
}

bool runs_resident(const lattice *lt)
{
    if (!resident_supported(lt->geom)) return false;
    if (choose_kernel(lt) == LAT_KERNEL_RESIDENT) return true;
    return lt->kernel == LAT_KERNEL_AUTO && lt->P.L <= kResidentMaxL;
}

// Launch the resident lattices on the side stream (after the work already
// on the batch stream) and record the join event.
int run_resident(lattice_batch *b, BatchSlot &sl, const std::vector<std::pair<lattice *, int64_t>> &res)
{
    const int n = (int)res.size();
    std::vector<Geom> geoms((size_t)n);
    std::vector<long long> counts((size_t)n);
    size_t smem = 0;
    long long most = 0;
    for (int i = 0; i < n; ++i) {
        geoms[(size_t)i] = tiled_geom(res[(size_t)i].first->geom);
        counts[(size_t)i] = (long long)res[(size_t)i].second;
        smem = std::max(smem, resident_smem_bytes(res[(size_t)i].first->geom));
        most = std::max(most, counts[(size_t)i]);
    }
    int rc = grow(&sl.d_res_geoms, sl.res_geoms_cap, n, b->stream);
    if (rc == LAT_OK) rc = grow(&sl.d_res_n, sl.res_n_cap, n, b->stream);
    if (rc == LAT_OK) rc = ensure_pinned(sl, (size_t)n * (sizeof(Geom) + sizeof(long long)) + 64);
    if (rc != LAT_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (b->res_stream == nullptr) e = cudaStreamCreateWithFlags(&b->res_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && b->ev_fork == nullptr) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && b->ev_join == nullptr) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    size_t at = 0;
    at = stage(sl, at, sl.d_res_geoms, geoms.data(), (size_t)n, b->stream, e);
    at = stage(sl, at, sl.d_res_n, counts.data(), (size_t)n, b->stream, e);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->res_stream, b->ev_fork, 0);
    for (long long done = 0; done < most && e == cudaSuccess; done += kResidentChunk)
        e = launch_batch_resident(sl.d_res_geoms, sl.d_res_n, n, done, kResidentChunk, smem, b->res_stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->res_stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch resident launch");
    return LAT_OK;
}

// The work lists of one phase (the first n_active lattices of `work`),
// appended to geoms / ctrls / items; returns its item counts.
Shape build_phase(const std::vector<std::pair<lattice *, int64_t>> &work, size_t n_active, int passes,
                  std::vector<Geom> &geoms, std::vector<Ctrl *> &ctrls, std::vector<uint2> &items)
{
    std::vector<uint2> tiled, tiled_ne, w2[3], grp[3], wide[2], potts, gen;
    int tab_gen = 0;
    // 3D / spin-S and Potts items: the rows per item follow the phase's whole
    // work of that kind (a few items per CTA), not the 2D tunable
    uint64_t chunk_rows3 = 0, chunk_rows_p = 0;
    for (size_t i = 0; i < n_active; ++i) {
        const lattice *lt = work[i].first;
        const int kern = choose_kernel(lt);
        const bool generic = kern == LAT_KERNEL_GENERIC;
        if (generic || (tiled_supported(lt->geom) && kern == LAT_KERNEL_TILED) || any_supported(lt->geom)) continue;
        const uint64_t cr = (uint64_t)lt->geom.rows * (lt->geom.half >> 3);
        if (wide3_supported(lt->geom)) chunk_rows3 += cr;
        else if (potts_supported(lt->geom)) chunk_rows_p += cr;
    }
    const int passes3 = batch_item_passes(chunk_rows3), passes_p = batch_item_passes(chunk_rows_p);
    for (size_t i = 0; i < n_active; ++i) {
        lattice *lt = work[i].first;
        geoms.push_back(tiled_geom(lt->geom));
        ctrls.push_back(lt->ctrl);
        // 2D spin-1/2 lattices take the tiled items when their kernel is the
        // tiled one, else the any-L items (16-byte aligned rows when
        // L % 32 == 0); 3D and spin-S Ising lattices with L % 16 == 0 take
        // the 3D wide items, Potts lattices with L % 16 == 0 the Potts items;
        // the rest (other sizes, per-site disorder, an explicit generic
        // choice) go to the generic chunks.  Item lattice indexes are local
        // to the phase.
        const int kern = choose_kernel(lt);
        const bool generic = kern == LAT_KERNEL_GENERIC;
        if (!generic && tiled_supported(lt->geom) && kern == LAT_KERNEL_TILED) {
            const int nt = tiles_of(lt->geom, 0);
            auto &dst = (lt->P.model == LAT_NE) ? tiled_ne : tiled;
            for (int k = 0; k < nt; ++k) dst.push_back(make_uint2((unsigned)i, (unsigned)k));
        } else if (!generic && any_supported(lt->geom)) {
            const int ng = any_items(lt->geom, passes);
            const int m = lt->P.model == LAT_NE ? (lt->geom.cmode ? 2 : 1) : 0;
            auto &dst = (lt->geom.L % 32 == 0 ? w2 : grp)[m];
            for (int k = 0; k < ng; ++k) dst.push_back(make_uint2((unsigned)i, (unsigned)k));
        } else if (!generic && wide3_supported(lt->geom)) {
            const int nw = wide3_items(lt->geom, passes3);
            auto &dst = wide[wide3_swar(lt->geom) ? 1 : 0];
            for (int k = 0; k < nw; ++k) dst.push_back(make_uint2((unsigned)i, (unsigned)k));
        } else if (!generic && potts_supported(lt->geom)) {
            const int np = potts_items(lt->geom, passes_p);
            for (int k = 0; k < np; ++k) potts.push_back(make_uint2((unsigned)i, (unsigned)k));
        } else {
            const uint64_t groups = (uint64_t)lt->geom.rows * lt->geom.G;
            const unsigned nc = (unsigned)((groups + kChunk - 1) / kChunk);
            for (unsigned k = 0; k < nc; ++k) gen.push_back(make_uint2((unsigned)i, k));
            tab_gen = std::max(tab_gen, lt->geom.tab_n);
        }
    }
    for (auto *v : {&tiled, &tiled_ne, &w2[0], &w2[1], &w2[2], &grp[0], &grp[1], &grp[2], &wide[0], &wide[1], &potts,
                    &gen})
        items.insert(items.end(), v->begin(), v->end());
    return Shape{(int)n_active, (int)tiled.size(), (int)tiled_ne.size(),
                 {(int)w2[0].size(), (int)w2[1].size(), (int)w2[2].size()},
                 {(int)grp[0].size(), (int)grp[1].size(), (int)grp[2].size()}, {(int)wide[0].size(), (int)wide[1].size()},
                 (int)potts.size(), (int)gen.size(), passes3, passes_p,
                 tab_gen};
}

// Upload a run's work lists into the slot's device arrays through its
// pinned staging, after the first res_bytes of staging (the resident
// lattices' uploads of the same run).
int upload_lists(lattice_batch *b, BatchSlot &sl, size_t res_bytes, const std::vector<Geom> &geoms,
                 const std::vector<uint2> &items, const std::vector<Ctrl *> &ctrls)
{
    int rc = grow(&sl.d_geoms, sl.geoms_cap, (int)geoms.size(), b->stream);
    if (rc == LAT_OK) rc = grow(&sl.d_items, sl.items_cap, (int)items.size(), b->stream);
    if (rc == LAT_OK) rc = grow(&sl.d_ctrls, sl.ctrls_cap, (int)ctrls.size(), b->stream);
    const size_t need = geoms.size() * sizeof(Geom) + items.size() * sizeof(uint2) + ctrls.size() * sizeof(Ctrl *) + 64;
    if (rc == LAT_OK && sl.h_cap < res_bytes + need) {
        // growing frees staging that earlier uploads of this run may still
        // read: wait for them first
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch staging");
        rc = ensure_pinned(sl, res_bytes + need);
    }
    if (rc != LAT_OK) return rc;
    cudaError_t e = cudaSuccess;
    size_t at = res_bytes;
    at = stage(sl, at, sl.d_geoms, geoms.data(), geoms.size(), b->stream, e);
    at = stage(sl, at, sl.d_items, items.data(), items.size(), b->stream, e);
    at = stage(sl, at, sl.d_ctrls, ctrls.data(), ctrls.size(), b->stream, e);
    if (e != cudaSuccess) return cuda_fail(e, "batch upload");
    return LAT_OK;
}

// Batch tuner: per composition of lattices (models, dimensions, spins,
// sizes and kernels of the lattices of a run's first phase), the rows per
// any-L item and the steps per captured graph, chosen by timing candidates
// on the run's own steps (one graph replay each after an untimed one; every
// candidate computes the same bits).  A run tunes only when its first phase
// has at least kBatchTuneMin steps (tuning synchronises the host, so short
// runs such as server rounds keep the defaults).  Choices last for the
// life of the process.
constexpr int64_t kBatchTuneMin = 192;
constexpr BatchTune kBatchCand[] = {{2, 8}, {2, 32}, {8, 8}, {8, 32}};   // 160 steps in all
std::mutex g_btune_mu;
std::map<uint64_t, BatchTune> g_btune;

uint64_t composition_key(const std::vector<std::pair<lattice *, int64_t>> &work)
{
    std::vector<uint64_t> v;
    v.reserve(work.size());
    for (auto &pr : work) {
        const lattice *lt = pr.first;
        v.push_back(((uint64_t)lt->P.model << 56) ^ ((uint64_t)lt->P.dims << 52) ^ ((uint64_t)lt->P.two_S << 44) ^
                    ((uint64_t)choose_kernel(lt) << 40) ^ ((uint64_t)(lt->geom.cpl != nullptr) << 39) ^
                    (uint64_t)lt->P.L);
    }
    std::sort(v.begin(), v.end());
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the sorted shape words
    for (uint64_t x : v)
        for (int k = 0; k < 8; ++k) {
            h ^= (x >> (8 * k)) & 0xFFu;
            h *= 1099511628211ull;
        }
    return h;
}

// Time the candidates on the first phase (all lattices of `work`); returns
// the steps run (every lattice advanced by them) and the pick.
int tune_batch(lattice_batch *b, BatchSlot &sl, size_t res_bytes, const std::vector<std::pair<lattice *, int64_t>> &work,
               int64_t &steps_run, BatchTune &pick)
{
    steps_run = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return cuda_fail(cudaGetLastError(), "batch tune");
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(cudaGetLastError(), "batch tune");
    }
    float best = 1e30f;
    int rc = LAT_OK;
    for (const BatchTune &c : kBatchCand) {
        std::vector<Geom> geoms;
        std::vector<Ctrl *> ctrls;
        std::vector<uint2> items;
        const Shape sh = build_phase(work, work.size(), c.passes, geoms, ctrls, items);
        rc = upload_lists(b, sl, res_bytes, geoms, items, ctrls);
        if (rc != LAT_OK) break;
        const Phase ph{sh, 2 * (int64_t)c.gsteps, sl.d_geoms, sl.d_items, sl.d_ctrls, c.passes, c.gsteps};
        cudaGraphExec_t exec = nullptr;
        rc = capture_steps(b, ph, c.gsteps, &exec);
        if (rc != LAT_OK) break;
        cudaError_t e = cudaGraphLaunch(exec, b->stream);   // untimed
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);   // the next candidate reuses the arrays
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "batch tune");
            break;
        }
        steps_run += 2 * c.gsteps;
        if (ms / c.gsteps < best) {
            best = ms / c.gsteps;
            pick = c;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return rc;
}

}  // namespace

extern "C" {

int lattice_batch_create(lattice_batch_t **out, void *cuda_stream)
{
    if (out == nullptr) return LAT_EINVAL;
    *out = nullptr;
    lattice_batch *b = new (std::nothrow) lattice_batch();
    if (b == nullptr) return LAT_ENOMEM;
    b->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = dev_alloc((void **)&b->d_counters, kCounters * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, kCounters * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) {
        delete b;
        return e == cudaErrorMemoryAllocation ? LAT_ENOMEM : cuda_fail(e, "batch create");
    }
    b->grid_tiled_ising = batch_tiled_grid(false);
    b->grid_tiled_ne = batch_tiled_grid(true);
    b->grid_generic = batch_generic_grid();
    b->grid_wide[0] = batch_wide3_grid(false);
    b->grid_wide[1] = batch_wide3_grid(true);
    b->grid_potts = batch_potts_grid();
    b->grid_any[0] = batch_any_grid(false);
    b->grid_any[1] = batch_any_grid(true);
    *out = b;
    return LAT_OK;
}

int lattice_batch_add(lattice_batch_t *b, lattice_t *lt, int64_t n)
{
    if (b == nullptr || lt == nullptr || n < 0) return LAT_EINVAL;
    if (lt->P.layout == LAT_BITPACKED || lt->dynamics != LAT_DYNAMICS_CHECKERBOARD) return LAT_ENOTSUP;
    if (n == 0) return LAT_OK;
    for (auto &pr : b->pending)
        if (pr.first == lt) {
            pr.second += n;
            return LAT_OK;
        }
    b->pending.emplace_back(lt, n);
    return LAT_OK;
}

int lattice_batch_run(lattice_batch_t *b)
{
    if (b == nullptr) return LAT_EINVAL;
    std::vector<std::pair<lattice *, int64_t>> work;
    work.swap(b->pending);
    if (work.empty()) return LAT_OK;
    // Counter space for every sweep of the run (queued on each lattice's own
    // stream), then the batch stream waits for the work queued so far on
    // each distinct lattice stream (lattices often share one): an event
    // wait, so the host does not block.
    std::vector<cudaStream_t> streams;
    for (auto &pr : work) {
        int rc = ensure_series(pr.first, (unsigned long long)(pr.first->sweeps + pr.second));
        if (rc != LAT_OK) return rc;
        cudaStream_t ls = pr.first->stream;
        if (ls != b->stream && std::find(streams.begin(), streams.end(), ls) == streams.end()) streams.push_back(ls);
    }
    while (b->ev_streams.size() < streams.size()) {
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "batch event");
        b->ev_streams.push_back(ev);
    }
    for (size_t i = 0; i < streams.size(); ++i) {
        cudaError_t e = cudaEventRecord(b->ev_streams[i], streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_streams[i], 0);
        if (e != cudaSuccess) return cuda_fail(e, "batch order");
    }
    BatchSlot *slp = nullptr;
    int rc0 = take_slot(b, &slp);
    if (rc0 != LAT_OK) return rc0;
    BatchSlot &sl = *slp;
    bool started = false;
    auto mark_start = [&]() {
        if (!started && b->start_event != nullptr) cudaEventRecord(b->start_event, b->stream);
        started = true;
    };
    // Small lattices: resident CTAs on the side stream.
    std::vector<std::pair<lattice *, int64_t>> res, rest;
    for (auto &pr : work) (runs_resident(pr.first) ? res : rest).push_back(pr);
    if (!res.empty()) {
        mark_start();
        int rc = run_resident(b, sl, res);
        if (rc != LAT_OK) return rc;
    }
    for (auto &pr : res) pr.first->sweeps += pr.second;
    work.swap(rest);
    // Run in phases: all lattices until the smallest remaining count is
    // done, then drop it, and so on.  Every phase's descriptors and items are
    // built first and uploaded together, so the phases are queued back to
    // back with no host synchronisation between them.
    std::sort(work.begin(), work.end(), [](const auto &a, const auto &c) { return a.second > c.second; });
    // the resident lattices' uploads sit at the front of the staging
    const size_t res_bytes =
        res.empty() ? 0 : ((res.size() * (sizeof(Geom) + sizeof(long long)) + 64 + 15) & ~(size_t)15);
    BatchTune tune{0, kGraphSteps};
    if (!work.empty()) {
        const uint64_t key = composition_key(work);
        bool found = false;
        {
            std::lock_guard<std::mutex> g(g_btune_mu);
            auto it = g_btune.find(key);
            if (it != g_btune.end()) {
                tune = it->second;
                found = true;
            }
        }
        if (!found && work.back().second >= kBatchTuneMin) {
            mark_start();
            int64_t steps_run = 0;
            int rc = tune_batch(b, sl, res_bytes, work, steps_run, tune);
            if (rc != LAT_OK) return rc;
            for (auto &pr : work) {   // the tuning steps were real steps of every lattice
                pr.second -= steps_run;
                pr.first->sweeps += steps_run;
            }
            std::lock_guard<std::mutex> g(g_btune_mu);
            g_btune[key] = tune;
        }
        b->last_passes = tune.passes;
        b->last_gsteps = tune.gsteps;
    }
    std::vector<Geom> all_geoms;
    std::vector<Ctrl *> all_ctrls;
    std::vector<uint2> all_items;
    struct Spec {
        Shape sh;
        int64_t steps;
        size_t geom_off, item_off;
    };
    std::vector<Spec> specs;
    int64_t done = 0;
    for (size_t n_active = work.size(); n_active > 0; --n_active) {
        const int64_t steps = work[n_active - 1].second - done;
        if (steps <= 0) continue;
        Spec sp;
        sp.geom_off = all_geoms.size();
        sp.item_off = all_items.size();
        sp.sh = build_phase(work, n_active, tune.passes, all_geoms, all_ctrls, all_items);
        sp.steps = steps;
        specs.push_back(sp);
        done += steps;
    }
    if (!specs.empty()) {
        int rc = upload_lists(b, sl, res_bytes, all_geoms, all_items, all_ctrls);
        if (rc != LAT_OK) return rc;
        mark_start();
        for (const Spec &sp : specs) {
            const Phase ph{sp.sh, sp.steps, sl.d_geoms + sp.geom_off, sl.d_items + sp.item_off,
                           sl.d_ctrls + sp.geom_off, tune.passes, tune.gsteps};
            rc = run_steps(b, ph);
            if (rc != LAT_OK) return rc;
        }
    }
    for (auto &pr : work) pr.first->sweeps += pr.second;
    mark_start();
    cudaError_t e = cudaSuccess;
    if (!res.empty()) e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    // Order later work on each lattice's own stream after the batch.
    if (e == cudaSuccess && b->ev_done == nullptr) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_done, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, b->stream);   // the slot is free again after this
    if (e == cudaSuccess) sl.used = true;
    if (!b->caller_orders) {
        streams.clear();
        for (auto *list : {&work, &res})
            for (auto &pr : *list) {
                cudaStream_t ls = pr.first->stream;
                if (ls != b->stream && std::find(streams.begin(), streams.end(), ls) == streams.end())
                    streams.push_back(ls);
            }
        for (cudaStream_t ls : streams)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ls, b->ev_done, 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch join");
    return LAT_OK;
}

}  // extern "C"

// The server orders every other use of its lattices against the batch
// stream itself (internal, not part of the C ABI).
void batch_set_caller_orders(lattice_batch_t *b, bool on)
{
    if (b) b->caller_orders = on;
}

void batch_set_start_event(lattice_batch_t *b, cudaEvent_t ev)
{
    if (b) b->start_event = ev;
}

extern "C" {

int lattice_batch_tuning(lattice_batch_t *b, int *rows_per_item, int *steps_per_graph)
{
    if (b == nullptr) return LAT_EINVAL;
    if (rows_per_item) *rows_per_item = b->last_passes;
    if (steps_per_graph) *steps_per_graph = b->last_gsteps;
    return LAT_OK;
}

int lattice_batch_synchronize(lattice_batch_t *b)
{
    if (b == nullptr) return LAT_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && b->res_stream) e = cudaStreamSynchronize(b->res_stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronize");
    return LAT_OK;
}

void lattice_batch_destroy(lattice_batch_t *b)
{
    if (b == nullptr) return;
    cudaStreamSynchronize(b->stream);
    if (b->res_stream) cudaStreamSynchronize(b->res_stream);
    for (BatchSlot &sl : b->slots) {
        dev_free(sl.d_geoms, b->stream);
        dev_free(sl.d_items, b->stream);
        dev_free(sl.d_ctrls, b->stream);
        dev_free(sl.d_res_geoms, b->stream);
        dev_free(sl.d_res_n, b->stream);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    cudaStreamSynchronize(b->stream);
    for (BatchSlot &sl : b->slots)
        if (sl.h_pin) cudaFreeHost(sl.h_pin);
    for (cudaEvent_t ev : b->ev_streams) cudaEventDestroy(ev);
    dev_free(b->d_counters, b->stream);
    if (b->res_stream) cudaStreamDestroy(b->res_stream);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

}  // extern "C"
