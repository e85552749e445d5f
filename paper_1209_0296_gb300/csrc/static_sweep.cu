// static_sweep.cu -- lattice_sweep_static: the batched tiled sweep for callers
// that cannot allocate device memory.
//
// Every other entry point of this library allocates: lattice_create owns
// its spin buffers, tables and counters, and the batch engine grows its
// work lists with cudaMallocAsync.  Some callers cannot let a library do
// that: a framework whose device memory all comes from its own caching pool
// (so that its accounting and fragmentation control stay exact), a
// memory-capped service that budgets every byte up front, or a
// latency-critical caller that must never hit the device-wide
// synchronisation a cudaMalloc / cudaFree can cause.  This entry point
// allocates nothing: the caller passes its own device buffers for the
// spins and the per-sweep counters, and the library's own scratch (lattice
// descriptors, acceptance tables, sweep-counter blocks and the tile work
// list) lives in the file-scope array below, which every GPU that loads
// the library holds until the process exits.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "lattice_capi_internal.h"

namespace lat {
namespace {

constexpr int kStaticMaxLattices = 64;
constexpr int kStaticMaxTiles = 65536;   // e.g. one L = 32768 lattice in 256 x 64 tiles
constexpr int kStaticTileH = 64;
constexpr int kTab2D = 45;               // (2*2+1) x (2*4+1) entries for 2D spin-1/2

struct StaticScratch {
    Geom geoms[kStaticMaxLattices];
    Ctrl ctrl[kStaticMaxLattices];
    Ctrl *ctrl_ptr[kStaticMaxLattices];
    TabEntry tab[kStaticMaxLattices][kTab2D];
    uint2 items[kStaticMaxTiles];
    unsigned next_item[4];
};

// The scratch: about 560 kB per device.  Host code must not use this name
// as an address (it is a host-side stand-in); the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) StaticScratch g_static_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
StaticScratch *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device with that device current.
int static_scratch(StaticScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return LAT_ERANGE;
    std::lock_guard<std::mutex> g(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_static_ptr[dev] = static_cast<StaticScratch *>(p);
    }
    *out = g_static_ptr[dev];
    return LAT_OK;
}

}  // namespace
}  // namespace lat

using namespace lat;

extern "C" int lattice_sweep_static(const lattice_static_desc_t *descs, int n_lattices, int64_t n_sweeps,
                                    void *cuda_stream)
{
    if (descs == nullptr || n_sweeps < 0) return LAT_EINVAL;
    if (n_lattices < 1 || n_lattices > kStaticMaxLattices) return LAT_ERANGE;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // Host-side descriptors (host memory only; nothing on the device yet).
    std::vector<Geom> geoms((size_t)n_lattices);
    std::vector<Ctrl> ctrls((size_t)n_lattices);
    std::vector<TabEntry> tabs((size_t)n_lattices * kTab2D);
    std::vector<uint2> items;
    for (int i = 0; i < n_lattices; ++i) {
        const lattice_static_desc_t &d = descs[i];
        Params P{};
        int rc = validate(2, d.L, 1, LAT_ISING, d.J, d.h, d.T, LAT_INIT_COLD, LAT_INT8, P);
        if (rc != LAT_OK) return rc;
        if (d.L % 32 != 0) return LAT_ENOTSUP;
        if (d.sweep0 < 0 || d.spins[0] == nullptr || d.spins[1] == nullptr ||
            (d.counters == nullptr && n_sweeps > 0))
            return LAT_EINVAL;
        std::vector<TabEntry> tab;
        int dsmax, nmax, nn;
        build_table(P, tab, dsmax, nmax, nn);
        if ((int)tab.size() != kTab2D) return LAT_ENOTSUP;
        Geom &g = geoms[(size_t)i];
        memset(&g, 0, sizeof g);
        g.dims = 2;
        g.L = d.L;
        g.two_S = 1;
        g.model = LAT_ISING;
        g.sh = 2;
        g.G = (uint32_t)(d.L / 8);
        g.rows = (uint32_t)d.L;
        g.N = P.N;
        g.key0 = (uint32_t)(d.seed & 0xffffffffu);
        g.key1 = (uint32_t)(d.seed >> 32);
        g.dsmax = dsmax;
        g.nmax = nmax;
        g.nn = nn;
        g.tab_n = kTab2D;
        g.s[0] = d.spins[0];
        g.s[1] = d.spins[1];
        g.half = (uint32_t)(d.L / 2);
        g.plane = P.N / 2;
        compact_table(g, tab.data());
        if (!tiled_supported(g)) return LAT_ENOTSUP;   // e.g. a never-accept table entry
        for (int k = 0; k < kTab2D; ++k) tabs[(size_t)i * kTab2D + k] = tab[(size_t)k];
        Ctrl &c = ctrls[(size_t)i];
        memset(&c, 0, sizeof c);
        c.sweep = (unsigned long long)d.sweep0;
        c.series = reinterpret_cast<unsigned long long *>(d.counters);
        c.series_base = (unsigned long long)d.sweep0;
        c.series_cap = (unsigned long long)n_sweeps;
        const int nt = tiles_of(g, kStaticTileH);
        if ((int64_t)items.size() + nt > kStaticMaxTiles) return LAT_ERANGE;
        for (int k = 0; k < nt; ++k) items.push_back(make_uint2((unsigned)i, (unsigned)k));
    }
    if (n_sweeps == 0) return LAT_OK;

    StaticScratch *sp = nullptr;
    int rc = static_scratch(&sp);
    if (rc != LAT_OK) return rc;
    // Point the descriptors at the scratch's tables and counter blocks.
    std::vector<Ctrl *> ctrl_ptrs((size_t)n_lattices);
    for (int i = 0; i < n_lattices; ++i) {
        geoms[(size_t)i].tab = &sp->tab[i][0];
        geoms[(size_t)i].ctrl = &sp->ctrl[i];
        geoms[(size_t)i] = tiled_geom(geoms[(size_t)i]);
        ctrl_ptrs[(size_t)i] = &sp->ctrl[i];
    }
    // Fill the scratch (it keeps the previous call's contents) and clear what
    // must start at zero: the item counters and the caller's counter slots.
    cudaError_t e = cudaMemcpyAsync(sp->geoms, geoms.data(), geoms.size() * sizeof(Geom),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sp->ctrl, ctrls.data(), ctrls.size() * sizeof(Ctrl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sp->ctrl_ptr, ctrl_ptrs.data(), ctrl_ptrs.size() * sizeof(Ctrl *),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sp->tab, tabs.data(), tabs.size() * sizeof(TabEntry), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sp->items, items.data(), items.size() * sizeof(uint2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sp->next_item, 0, sizeof sp->next_item, st);
    for (int i = 0; i < n_lattices && e == cudaSuccess; ++i)
        e = cudaMemsetAsync(descs[i].counters, 0, (size_t)n_sweeps * 4 * sizeof(int64_t), st);
    // The host vectors above are released on return: let the copies finish.
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "static sweep set-up");
    const int grid = std::min(batch_tiled_grid(false), (int)items.size());
    for (int64_t s = 0; s < n_sweeps; ++s) {
        e = launch_batch_tiled(sp->geoms, sp->items, (int)items.size(), &sp->next_item[0], kStaticTileH, 0,
                               grid, false, st);
        if (e == cudaSuccess) e = launch_batch_advance(sp->ctrl_ptr, n_lattices, sp->next_item, 1, 1ull, st);
        if (e != cudaSuccess) return cuda_fail(e, "static sweep launch");
    }
    return LAT_OK;
}
