// server.cu -- lattice_server_*: continuous batching of independent
// simulation requests on one GPU.
//
// One scheduler thread owns a CUDA stream and a lattice_batch.  Requests
// wait in arrival order; between scheduling rounds the scheduler admits as
// many as fit (device footprint within the HBM budget, resident count below
// max_slots), creates their lattices on the device, then runs one round:
// every resident lattice advances by min(chunk, remaining) sweeps in shared
// batched launches.  Lattices that are done are read back (counters,
// observables, optionally spins) and destroyed, which frees budget for the
// next admissions.  Requests therefore join and leave while others keep
// running, and each result is the same as its lattice alone (the batch
// engine is bit-exact per lattice).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lattice_capi_internal.h"

using namespace lat;

namespace {

struct Req {
    uint64_t id;
    lattice_request_t r;
    Params P;
    size_t bytes;          // device footprint charged against the budget
    lattice *lt = nullptr;
    int64_t done = 0;      // sweeps completed
    lattice_result_t res{};
    std::vector<int8_t> spins;
};

}  // namespace

struct lattice_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> waiting;
    std::vector<Req *> resident;
    std::unordered_map<uint64_t, Req *> all;   // submitted and not yet released
    uint64_t next_id = 1;
    size_t budget = 0, used = 0;
    int max_slots = 0, chunk = 0;
    bool stop = false;
    int device = 0;
    int64_t unfinished = 0;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    cudaStream_t stream = nullptr;
    lattice_batch_t *batch = nullptr;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

size_t request_bytes(const Params &P, int64_t sweeps)
{
    return footprint_bytes(P) + (size_t)(sweeps + 64) * 4 * sizeof(long long) * 2;
}

void finish(lattice_server *s, Req *q, int status)
{
    q->res.status = status;
    q->res.sweeps_done = q->done;
    q->res.t_done = s->now();
}

// Read the final counters (and spins) of a finished lattice, then free it.
void retire(lattice_server *s, Req *q)
{
    int rc = LAT_OK;
    if (q->done > 0) {
        int64_t b, m, u, f;
        rc = lattice_series(q->lt, q->done - 1, 1, &b, &m, &u, &f);
        if (rc == LAT_OK) {
            q->res.bond = b;
            q->res.mag = m;
            q->res.up = u;
            q->res.unflipped = f;
        }
    }
    if (rc == LAT_OK)
        rc = lattice_observables(q->lt, &q->res.E, &q->res.M, &q->res.density, &q->res.persistence);
    if (rc == LAT_OK && q->r.keep_spins) {
        q->spins.resize((size_t)q->P.N);
        rc = lattice_get_spins(q->lt, q->spins.data());
    }
    lattice_destroy(q->lt);
    q->lt = nullptr;
    std::lock_guard<std::mutex> g(s->mu);
    s->used -= q->bytes;
    finish(s, q, rc);
    --s->unfinished;
    s->cv_done.notify_all();
}

void scheduler(lattice_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        // ---- admission (arrival order; stop at the first that does not fit)
        std::vector<Req *> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->waiting.empty() || !s->resident.empty(); });
            if (s->stop) return;
            while (!s->waiting.empty()) {
                Req *q = s->waiting.front();
                if ((int)(s->resident.size() + admit.size()) >= s->max_slots) break;
                if (s->used + q->bytes > s->budget) break;
                s->waiting.pop_front();
                s->used += q->bytes;
                admit.push_back(q);
            }
        }
        for (Req *q : admit) {
            q->res.t_admit = s->now();
            const lattice_request_t &r = q->r;
            int rc = create_impl(&q->lt, r.dims, r.L, r.two_S, r.model, r.J, r.h, r.T_or_c, r.seed,
                                 r.init, LAT_INT8, s->stream);
            std::lock_guard<std::mutex> g(s->mu);
            if (rc != LAT_OK) {
                s->used -= q->bytes;
                finish(s, q, rc);
                --s->unfinished;
                s->cv_done.notify_all();
            } else {
                s->resident.push_back(q);  // (0 sweeps: retired after this round)
            }
        }
        // ---- one round over the resident lattices
        std::vector<Req *> res;
        {
            std::lock_guard<std::mutex> g(s->mu);
            res = s->resident;
        }
        int rc = LAT_OK;
        for (Req *q : res) {
            const int64_t k = std::min<int64_t>(s->chunk, q->r.sweeps - q->done);
            if (k > 0) rc = lattice_batch_add(s->batch, q->lt, k);
            if (rc != LAT_OK) break;
        }
        if (rc == LAT_OK) rc = lattice_batch_run(s->batch);
        if (rc == LAT_OK) rc = lattice_batch_synchronize(s->batch);
        std::vector<Req *> keep, out;
        for (Req *q : res) {
            if (rc != LAT_OK) {
                out.push_back(q);
                continue;
            }
            q->done += std::min<int64_t>(s->chunk, q->r.sweeps - q->done);
            (q->done >= q->r.sweeps ? out : keep).push_back(q);
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->resident = keep;
        }
        for (Req *q : out) {
            if (rc != LAT_OK) {
                lattice_destroy(q->lt);
                q->lt = nullptr;
                std::lock_guard<std::mutex> g(s->mu);
                s->used -= q->bytes;
                finish(s, q, rc);
                --s->unfinished;
                s->cv_done.notify_all();
            } else {
                retire(s, q);
            }
        }
    }
}

}  // namespace

extern "C" {

int lattice_server_create(lattice_server_t **out, size_t hbm_budget_bytes, int max_slots, int chunk_sweeps)
{
    if (out == nullptr || hbm_budget_bytes == 0 || max_slots < 1 || chunk_sweeps < 1) return LAT_EINVAL;
    *out = nullptr;
    lattice_server *s = new (std::nothrow) lattice_server();
    if (s == nullptr) return LAT_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->chunk = chunk_sweeps;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "server create");
    }
    int rc = lattice_batch_create(&s->batch, s->stream);
    if (rc != LAT_OK) {
        cudaStreamDestroy(s->stream);
        delete s;
        return rc;
    }
    try {
        s->worker = std::thread(scheduler, s);
    } catch (...) {
        lattice_batch_destroy(s->batch);
        cudaStreamDestroy(s->stream);
        delete s;
        return LAT_ENOMEM;
    }
    *out = s;
    return LAT_OK;
}

int lattice_server_submit(lattice_server_t *s, const lattice_request_t *req, uint64_t *id)
{
    if (s == nullptr || req == nullptr || id == nullptr || req->sweeps < 0) return LAT_EINVAL;
    Params P{};
    int rc = validate(req->dims, req->L, req->two_S, req->model, req->J, req->h, req->T_or_c, req->init,
                      LAT_INT8, P);
    if (rc != LAT_OK) return rc;
    const size_t bytes = request_bytes(P, req->sweeps);
    if (bytes > s->budget) return LAT_ENOMEM;   // could never be admitted
    Req *q = new (std::nothrow) Req();
    if (q == nullptr) return LAT_ENOMEM;
    q->r = *req;
    q->P = P;
    q->bytes = bytes;
    std::lock_guard<std::mutex> g(s->mu);
    q->id = s->next_id++;
    q->res.status = LAT_EBUSY;
    q->res.t_submit = s->now();
    s->all[q->id] = q;
    s->waiting.push_back(q);
    ++s->unfinished;
    *id = q->id;
    s->cv_work.notify_one();
    return LAT_OK;
}

int lattice_server_poll(lattice_server_t *s, uint64_t id, lattice_result_t *res, int8_t *spins_out)
{
    if (s == nullptr) return LAT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LAT_ENOENT;
    Req *q = it->second;
    if (q->res.status == LAT_EBUSY) return LAT_EBUSY;
    if (res) *res = q->res;
    if (spins_out != nullptr && !q->spins.empty()) memcpy(spins_out, q->spins.data(), q->spins.size());
    s->all.erase(it);
    delete q;
    return LAT_OK;
}

int lattice_server_drain(lattice_server_t *s, double timeout_s)
{
    if (s == nullptr) return LAT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] { return s->unfinished == 0; };
    if (timeout_s <= 0) {
        s->cv_done.wait(lk, done);
        return LAT_OK;
    }
    return s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done) ? LAT_OK : LAT_ETIMEOUT;
}

double lattice_server_clock(lattice_server_t *s) { return s ? s->now() : 0.0; }

void lattice_server_destroy(lattice_server_t *s)
{
    if (s == nullptr) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    s->worker.join();
    for (Req *q : s->resident)
        if (q->lt) lattice_destroy(q->lt);
    for (auto &kv : s->all) delete kv.second;
    lattice_batch_destroy(s->batch);
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
