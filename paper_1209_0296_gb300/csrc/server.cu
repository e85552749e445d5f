// server.cu -- lattice_server_*: continuous batching of independent
// simulation requests on one GPU.
//
// One scheduler thread owns a CUDA stream and a lattice_batch.  Requests
// wait in arrival order and are admitted as far as the HBM budget and the
// slot limit allow; their lattices are created on a second stream (the
// creation stream), with counter space for all their sweeps.  Each
// scheduling round advances every resident lattice by min(chunk,
// remaining) sweeps in shared batched launches.  Rounds are pipelined: the
// scheduler queues round k+1 while round k runs, and a lattice whose last
// sweep is in round k is retired (counters, observables and optionally
// spins read back on the creation stream, memory freed) once round k's
// event has completed -- so admission, creation and retirement overlap the
// device's work instead of leaving it idle.  Requests therefore join and
// leave while others keep running, and each result is the same as its
// lattice alone (the batch engine is bit-exact per lattice).  A request
// whose creation or queueing fails ends with that error alone; only a
// failed launch (a CUDA error) ends every request of its round.
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

// batch.cu: the server orders every other use of its lattices itself, and
// reads the start of each run's device work from an event
void batch_set_caller_orders(lattice_batch_t *b, bool on);
void batch_set_start_event(lattice_batch_t *b, cudaEvent_t ev);

namespace {

struct Req {
    uint64_t id;
    lattice_request_t r;
    Params P;
    size_t bytes;          // device footprint charged against the budget
    lattice *lt = nullptr;
    int64_t planned = 0;   // sweeps queued so far
    lattice_result_t res{};
    std::vector<int8_t> spins;
};

// A queued round: its completion event, its timing events and the
// requests whose last sweep it runs.
struct Round {
    cudaEvent_t done = nullptr, t_start = nullptr, t_end = nullptr;
    std::vector<Req *> retiring;
    std::vector<Req *> members;   // every request with work in the round
    bool failed = false;
    int rc = LAT_OK;
};

}  // namespace

struct lattice_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> waiting;
    std::vector<Req *> resident;              // admitted, sweeps left to queue
    std::unordered_map<uint64_t, Req *> all;   // submitted and not yet released
    uint64_t next_id = 1;
    size_t budget = 0, used = 0;
    int max_slots = 0, chunk = 0;
    int in_device = 0;                         // admitted and not yet retired
    bool stop = false;
    int device = 0;
    int64_t unfinished = 0;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    cudaStream_t stream = nullptr;             // batched rounds
    cudaStream_t create_stream = nullptr;      // lattice creation, read-back, release
    lattice_batch_t *batch = nullptr;
    // statistics: device time of the rounds, rounds run
    double busy_s = 0.0;
    int64_t rounds = 0;

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

// Under s->mu.
void finish_locked(lattice_server *s, Req *q, int status)
{
    q->res.status = status;
    q->res.sweeps_done = status == LAT_OK ? q->r.sweeps : 0;
    q->res.t_done = s->now();
    s->used -= q->bytes;
    --s->in_device;
    --s->unfinished;
    s->cv_done.notify_all();
}

void fail(lattice_server *s, Req *q, int status)
{
    if (q->lt) {
        lattice_destroy(q->lt);
        q->lt = nullptr;
    }
    std::lock_guard<std::mutex> g(s->mu);
    finish_locked(s, q, status);
}

// Read the final counters (and spins) of a lattice whose last round has
// completed, then free it.  Everything here runs on the creation stream,
// which the batch never makes wait on later rounds.
void retire(lattice_server *s, Req *q)
{
    int rc = LAT_OK;
    if (q->r.sweeps > 0) {
        int64_t b, m, u, f;
        rc = lattice_series(q->lt, q->r.sweeps - 1, 1, &b, &m, &u, &f);
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
    finish_locked(s, q, rc);
}

void close_round(lattice_server *s, Round &rd)
{
    if (!rd.failed) {
        float ms = 0.0f;
        // (both timing events are recorded only when the round had work)
        if (!rd.members.empty() && cudaEventElapsedTime(&ms, rd.t_start, rd.t_end) == cudaSuccess)
            s->busy_s += ms * 1e-3;
        ++s->rounds;
        for (Req *q : rd.retiring) retire(s, q);
    } else {
        for (Req *q : rd.retiring) fail(s, q, rd.rc);
    }
    cudaEventDestroy(rd.done);
    cudaEventDestroy(rd.t_start);
    cudaEventDestroy(rd.t_end);
}

// Create the lattices of newly admitted requests (on the creation stream,
// with counter space for all their sweeps); a failure ends that request only.
void create_admitted(lattice_server *s, std::vector<Req *> &admit)
{
    for (Req *q : admit) {
        q->res.t_admit = s->now();
        const lattice_request_t &r = q->r;
        int rc = create_impl(&q->lt, r.dims, r.L, r.two_S, r.model, r.J, r.h, r.T_or_c, r.seed, r.init, LAT_INT8,
                             s->create_stream);
        if (rc == LAT_OK) rc = ensure_series(q->lt, (unsigned long long)r.sweeps);
        if (rc == LAT_OK) {
            cudaError_t e = cudaStreamSynchronize(s->create_stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "server create");
        }
        if (rc != LAT_OK) {
            fail(s, q, rc);
            continue;
        }
        std::lock_guard<std::mutex> g(s->mu);
        s->resident.push_back(q);
    }
}

void scheduler(lattice_server *s)
{
    cudaSetDevice(s->device);
    std::deque<Round> inflight;
    for (;;) {
        // ---- retire rounds that have completed; keep at most two queued
        while (!inflight.empty()) {
            Round &rd = inflight.front();
            bool block;
            {
                std::lock_guard<std::mutex> g(s->mu);
                // block when two rounds are queued, or when nothing else can
                // be done until the oldest completes
                block = inflight.size() >= 2 || (s->resident.empty() &&
                                                 (s->waiting.empty() || (int)s->in_device >= s->max_slots ||
                                                  s->used + s->waiting.front()->bytes > s->budget));
            }
            const cudaError_t e = block ? cudaEventSynchronize(rd.done) : cudaEventQuery(rd.done);
            if (e == cudaErrorNotReady) {
                (void)cudaGetLastError();   // "not ready" is no error: leave no trace for later launch checks
                break;
            }
            if (e != cudaSuccess) {
                rd.failed = true;
                rd.rc = cuda_fail(e, "server round");
            }
            close_round(s, rd);
            inflight.pop_front();
        }
        // ---- admission (arrival order; stop at the first that does not fit)
        std::vector<Req *> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (inflight.empty())
                s->cv_work.wait(lk, [&] { return s->stop || !s->waiting.empty() || !s->resident.empty(); });
            if (s->stop) break;
            while (!s->waiting.empty()) {
                Req *q = s->waiting.front();
                if (s->in_device >= s->max_slots) break;
                if (s->used + q->bytes > s->budget) break;
                s->waiting.pop_front();
                s->used += q->bytes;
                ++s->in_device;
                admit.push_back(q);
            }
        }
        create_admitted(s, admit);
        // ---- queue one round over the resident lattices
        std::vector<Req *> res;
        {
            std::lock_guard<std::mutex> g(s->mu);
            res.swap(s->resident);
        }
        if (res.empty()) continue;
        Round rd;
        std::vector<Req *> keep;
        for (Req *q : res) {
            const int64_t k = std::min<int64_t>(s->chunk, q->r.sweeps - q->planned);
            if (k > 0) {
                const int rc = lattice_batch_add(s->batch, q->lt, k);
                if (rc != LAT_OK) {   // this request alone
                    fail(s, q, rc);
                    continue;
                }
                q->planned += k;
                rd.members.push_back(q);
            }
            (q->planned >= q->r.sweeps ? rd.retiring : keep).push_back(q);
        }
        cudaError_t e = cudaEventCreateWithFlags(&rd.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&rd.t_start);
        if (e == cudaSuccess) e = cudaEventCreate(&rd.t_end);
        int rc = e == cudaSuccess ? LAT_OK : cuda_fail(e, "server events");
        batch_set_start_event(s->batch, rd.t_start);
        if (rc == LAT_OK) rc = lattice_batch_run(s->batch);
        batch_set_start_event(s->batch, nullptr);
        if (rc == LAT_OK) {
            e = cudaEventRecord(rd.t_end, s->stream);
            if (e == cudaSuccess) e = cudaEventRecord(rd.done, s->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "server round");
        }
        if (rc != LAT_OK) {
            // a failed launch: every request with work in this round ends
            // with the error (the device state of their lattices is unknown)
            for (Req *q : rd.members)
                if (std::find(rd.retiring.begin(), rd.retiring.end(), q) == rd.retiring.end()) {
                    keep.erase(std::remove(keep.begin(), keep.end(), q), keep.end());
                    rd.retiring.push_back(q);
                }
            cudaStreamSynchronize(s->stream);
            rd.failed = true;
            rd.rc = rc;
            if (rd.done == nullptr) cudaEventCreateWithFlags(&rd.done, cudaEventDisableTiming);
            cudaEventRecord(rd.done, s->stream);
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->resident.insert(s->resident.begin(), keep.begin(), keep.end());
        }
        inflight.push_back(std::move(rd));
    }
    // stopping: finish what is queued
    for (Round &rd : inflight) {
        cudaEventSynchronize(rd.done);
        close_round(s, rd);
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
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->create_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return cuda_fail(e, "server create");
    }
    int rc = lattice_batch_create(&s->batch, s->stream);
    if (rc != LAT_OK) {
        cudaStreamDestroy(s->stream);
        cudaStreamDestroy(s->create_stream);
        delete s;
        return rc;
    }
    batch_set_caller_orders(s->batch, true);
    try {
        s->worker = std::thread(scheduler, s);
    } catch (...) {
        lattice_batch_destroy(s->batch);
        cudaStreamDestroy(s->stream);
        cudaStreamDestroy(s->create_stream);
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
    cudaStreamSynchronize(s->stream);
    for (Req *q : s->resident)
        if (q->lt) lattice_destroy(q->lt);
    for (auto &kv : s->all) delete kv.second;
    lattice_batch_destroy(s->batch);
    cudaStreamSynchronize(s->create_stream);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->create_stream);
    delete s;
}

int lattice_server_stats(lattice_server_t *s, double *busy_s, double *wall_s, int64_t *rounds)
{
    if (s == nullptr) return LAT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (busy_s) *busy_s = s->busy_s;
    if (wall_s) *wall_s = s->now();
    if (rounds) *rounds = s->rounds;
    return LAT_OK;
}

}  // extern "C"
