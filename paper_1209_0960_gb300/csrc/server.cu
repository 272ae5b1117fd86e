// Serving: many independent AMG-PCG solves with continuous batching.
//
// Request life cycle (all times on the host steady clock):
//   queued   -> admitted when a slot is free and its device-memory estimate
//               fits the budget (FIFO, so a large request is not starved);
//   setup    -> a setup thread runs amg_setup (host aggregation, colouring,
//               then the GPU Galerkin products and level build on the
//               request's own stream) and replaces the estimate by the bytes
//               the hierarchy actually holds;
//   running  -> the scheduling thread uploads b, starts the CG and then
//               advances it one step at a time, for every running request in
//               turn, never blocking on any of them.  With batch_vcycles (the
//               default) every scheduler tick collects the requests whose
//               next step needs a preconditioner application and runs their
//               V-cycles together, level by level: each step of the V-cycle
//               (a colour pass, a residual, a restriction, a prolongation, a
//               coarsest solve) is one launch over all those requests
//               (batched_precondition), ordered after each request's previous
//               work by events, and each request's CG vector work follows on
//               its own stream.  Without it each request issues its own
//               launches (pcg_async_step), which overlap in the device queues;
//   draining -> the solution is copied back to pinned host memory;
//   done     -> the context is freed (stream-ordered, no device-wide
//               synchronisation), the slot and memory go to the next queued
//               request, and amg_poll hands the result out.
// A request's rows are computed by exactly the kernel bodies amg_setup +
// amg_pcg_solve use for it alone (a batched launch runs each request's
// segment as its own launch would), so its result does not depend on what
// else is in flight.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "device.h"

namespace amg {
extern thread_local std::string t_last_error;
}

using namespace amg;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    enum State { kQueued, kSetup, kReady, kSolving, kDraining, kDone };
    uint64_t ticket = 0;
    int32_t n = 0, nnz = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> va, b, x;
    double tol = 0.0;
    State state = kQueued;
    int status = AMG_OK;
    std::string error;
    amg_solve_info info{};
    amg_ctx* ctx = nullptr;
    double* pin = nullptr;     // pinned staging of b, then of x
    double hbm = 0.0;          // bytes reserved against the budget
    bool batch_failed = false; // its batched V-cycle could not be issued
    Clock::time_point t_submit, t_admit, t_ready, t_done;
};

}  // namespace

struct amg_server {
    amg_server_params p{};
    int device = 0;
    cudaStream_t batch_stream = nullptr;   // the batched V-cycles
    cudaEvent_t batch_ev = nullptr;        // the last batched V-cycle has been issued
    std::mutex mu;
    std::condition_variable cv_worker, cv_setup;
    std::deque<Request*> queued, setup_q, ready_q;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<Request*> running;   // owned by the scheduling thread
    std::vector<Request*> want;      // this tick: requests whose next step needs z = B r
    std::vector<int> want_first;     // ... and whether it is their first direction
    int64_t batches = 0, batched_requests = 0;
    bool stopping = false;
    double budget = 0.0, reserved = 0.0;
    int admitted = 0;                // requests in setup or running
    int setups_in_flight = 0;
    uint64_t next_ticket = 1;
    int64_t n_submitted = 0, n_completed = 0, n_failed = 0;
    int peak_running = 0;
    std::thread worker;
    std::vector<std::thread> setup_pool;
};

namespace {

// Device bytes a request will hold (hierarchy in float64 and float32, CG and
// level vectors, the dense coarsest inverse and its scaled copy) plus the
// setup-time copy of the matrix; refined after setup.
double estimate_bytes(const amg_server* S, const Request* r) {
    const double ct = std::min<double>(S->p.params.coarsen_target, S->p.params.dense_cap);
    return 1.4 * (36.0 * r->nnz + 160.0 * r->n) + 16.0 * ct * ct;
}

// Under the lock: admit queued requests in order while a slot and memory are
// free (an idle server always admits the head request, so one request larger
// than the budget still runs, and fails cleanly if memory runs out).
void admit_locked(amg_server* S) {
    while (!S->queued.empty() && S->admitted < S->p.max_slots) {
        Request* r = S->queued.front();
        const double est = estimate_bytes(S, r);
        if (S->admitted > 0 && S->reserved + est > S->budget) break;
        S->queued.pop_front();
        r->hbm = est;
        S->reserved += est;
        S->admitted += 1;
        S->peak_running = std::max(S->peak_running, S->admitted);
        r->state = Request::kSetup;
        r->t_admit = Clock::now();
        S->setup_q.push_back(r);
        S->cv_setup.notify_one();
    }
}

// Under the lock: a request leaves the device.
void finish_locked(amg_server* S, Request* r) {
    S->reserved -= r->hbm;
    S->admitted -= 1;
    r->state = Request::kDone;
    r->t_done = Clock::now();
    if (r->status == AMG_OK) S->n_completed += 1;
    else S->n_failed += 1;
}

void setup_main(amg_server* S) {
    cudaSetDevice(S->device);
    while (true) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_setup.wait(lk, [&] { return S->stopping || !S->setup_q.empty(); });
            if (S->setup_q.empty()) return;
            r = S->setup_q.front();
            S->setup_q.pop_front();
            S->setups_in_flight += 1;
        }
        amg_csr A{r->n, r->nnz, r->rp.data(), r->ci.data(), r->va.data(), 0};
        amg_params prm = S->p.params;
        prm.cuda_stream = nullptr;
        amg_ctx* c = nullptr;
        int rc = amg_setup(&A, &prm, &c);
        std::string err = rc == AMG_OK ? std::string() : std::string(amg_last_error());
        double* pin = nullptr;
        if (rc == AMG_OK) {
            try {
                pin = static_cast<double*>(pinned_alloc(sizeof(double) * (size_t)r->n));
            } catch (const Error& e) {
                rc = e.code;
                err = e.msg;
                amg_free(c);
                c = nullptr;
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->setups_in_flight -= 1;
            if (rc != AMG_OK) {
                r->status = rc;
                r->error = err;
                finish_locked(S, r);
            } else {
                const double actual = (double)c->mem.bytes();
                S->reserved += actual - r->hbm;
                r->hbm = actual;
                r->ctx = c;
                r->pin = pin;
                r->state = Request::kReady;
                r->t_ready = Clock::now();
                S->ready_q.push_back(r);
            }
            admit_locked(S);
        }
        S->cv_worker.notify_one();
    }
}

bool batched(const amg_server* S) { return S->p.batch_vcycles && !S->p.params.device_loop; }

// Issue the tick's batched V-cycle for the collected requests, each ordered
// after its own stream's work, then each request's rest of the iteration on
// its own stream after the batch.  Requests whose levels run sweep kernels
// (cooperative launches) precondition on their own streams.
void run_batch(amg_server* S, bool& progress) {
    std::vector<Request*>& w = S->want;
    if (w.empty()) return;
    progress = true;
    std::vector<amg_ctx*> cs;
    std::vector<size_t> own;
    for (size_t k = 0; k < w.size(); ++k) {
        amg_ctx* c = w[k]->ctx;
        bool ok = true;
        for (const DevLevel& L : c->dl) ok = ok && !L.sweep;
        if (!ok) own.push_back(k);
        else cs.push_back(c);
    }
    if (cs.size() == 1) {
        // a batch of one: its own launches on its own stream (the same bodies,
        // no cross-stream events)
        for (size_t k = 0; k < w.size(); ++k)
            if (w[k]->ctx == cs[0]) own.push_back(k);
        cs.clear();
    }
    for (amg_ctx* c : cs) {
        AMG_CUDA_TRY(cudaEventRecord(c->acg.ev, c->stream));
        AMG_CUDA_TRY(cudaStreamWaitEvent(S->batch_stream, c->acg.ev, 0));
    }
    if (!cs.empty()) {
        t_launch_overlap = S->p.params.launch_overlap != 0;
        batched_precondition(cs.data(), (int)cs.size(), S->batch_stream);
        AMG_CUDA_TRY(cudaEventRecord(S->batch_ev, S->batch_stream));
    }
    for (size_t k = 0; k < w.size(); ++k) {
        amg_ctx* c = w[k]->ctx;
        const bool mine = std::find(own.begin(), own.end(), k) != own.end();
        if (mine) {
            t_launch_overlap = c->p.launch_overlap != 0;
            precondition_context(c);
        } else {
            AMG_CUDA_TRY(cudaStreamWaitEvent(c->stream, S->batch_ev, 0));
        }
        pcg_async_resume(c, S->want_first[k] != 0);
    }
    if (!cs.empty()) {
        S->batches += 1;
        S->batched_requests += (int64_t)cs.size();
    }
    w.clear();
    S->want_first.clear();
}

// Advance one running request; returns true when it has left the device.
// `progress` is set when anything was issued or completed.
bool drive(amg_server* S, Request* r, bool& progress) {
    amg_ctx* c = r->ctx;
    const int n = r->n;
    try {
        switch (r->state) {
            case Request::kReady: {
                t_launch_overlap = c->p.launch_overlap != 0;
                std::memcpy(r->pin, r->b.data(), sizeof(double) * n);
                AMG_CUDA_TRY(cudaMemcpyAsync(c->q, r->pin, sizeof(double) * n,
                                             cudaMemcpyHostToDevice, c->stream));
                launch_scatter(n, c->perm0, c->q, c->bb, c->stream);
                AMG_CUDA_TRY(cudaMemsetAsync(c->x, 0, sizeof(double) * n, c->stream));
                pcg_async_begin(c, r->tol, S->p.maxit);
                r->state = Request::kSolving;
                progress = true;
                return false;
            }
            case Request::kSolving: {
                int st;
                if (batched(S)) {
                    bool first = false;
                    st = pcg_async_poll(c, &first);
                    if (st == 3) {
                        // next step needs z = B r: join this tick's batch
                        S->want.push_back(r);
                        S->want_first.push_back(first ? 1 : 0);
                        return false;
                    }
                } else {
                    st = pcg_async_step(c);
                }
                if (st == 0) return false;
                progress = true;
                if (st == 2) {
                    t_launch_overlap = c->p.launch_overlap != 0;
                    launch_gather(n, c->perm0, c->x, c->z, c->stream);
                    AMG_CUDA_TRY(cudaMemcpyAsync(r->pin, c->z, sizeof(double) * n,
                                                 cudaMemcpyDeviceToHost, c->stream));
                    AMG_CUDA_TRY(cudaEventRecord(c->acg.ev, c->stream));
                    r->state = Request::kDraining;
                }
                return false;
            }
            case Request::kDraining: {
                if (r->batch_failed) break;
                const cudaError_t q = cudaEventQuery(c->acg.ev);
                if (q == cudaErrorNotReady) return false;
                AMG_CUDA_TRY(q);
                r->x.assign(r->pin, r->pin + n);
                r->info = c->acg.info;
                r->status = c->acg.status;
                break;
            }
            default:
                return false;
        }
    } catch (const Error& e) {
        r->status = e.code;
        r->error = e.msg;
    }
    // leave the device: stream-ordered frees, pinned buffer back to the pool
    progress = true;
    amg_free(c);
    r->ctx = nullptr;
    pinned_free(r->pin);
    r->pin = nullptr;
    r->b.clear();
    r->b.shrink_to_fit();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        finish_locked(S, r);
        admit_locked(S);
    }
    return true;
}

void worker_main(amg_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*>& run = S->running;
    int idle = 0;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            admit_locked(S);
            while (!S->ready_q.empty()) {
                run.push_back(S->ready_q.front());
                S->ready_q.pop_front();
            }
            if (run.empty()) {
                if (S->stopping && S->setup_q.empty() && S->setups_in_flight == 0) break;
                S->cv_worker.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        bool progress = false;
        for (size_t i = 0; i < run.size();) {
            if (drive(S, run[i], progress)) run.erase(run.begin() + (long)i);
            else ++i;
        }
        try {
            run_batch(S, progress);
        } catch (const Error& e) {
            // a failed batch fails its requests (their contexts are freed on the next drive)
            for (Request* r : S->want) {
                r->status = e.code;
                r->error = e.msg;
                r->state = Request::kDraining;
                r->batch_failed = true;
            }
            S->want.clear();
            S->want_first.clear();
        }
        if (progress) {
            idle = 0;
        } else if (++idle > 2000) {
            // nothing completed for a while (long iterations): poll less often
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_worker.wait_for(lk, std::chrono::microseconds(200));
        } else {
            std::this_thread::yield();
        }
    }
}

template <typename F>
int guarded(F&& f) {
    try {
        f();
        t_last_error.clear();
        return AMG_OK;
    } catch (const Error& e) {
        t_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        t_last_error = "host allocation failed";
        return AMG_ENOMEM;
    } catch (const std::exception& e) {
        t_last_error = e.what();
        return AMG_EINVAL;
    }
}

}  // namespace

extern "C" {

int amg_server_params_default(amg_server_params* p, int32_t dim) {
    if (!p) return AMG_EINVAL;
    std::memset(p, 0, sizeof(*p));
    const int rc = amg_params_default(&p->params, dim);
    if (rc != AMG_OK) return rc;
    p->params.precision = AMG_FP32_IN_FP64;
    p->params.coarsen_target = 1000;
    // host-stepped iterations: with many solves sharing the GPU, the per-request
    // capture of the whole-loop graph cost more than the per-iteration events
    p->params.device_loop = 0;
    p->max_slots = 32;
    p->setup_threads = 4;
    p->maxit = 500;
    p->hbm_budget_bytes = 0.0;
    // measured on the 400-request serving stream: batching the V-cycles of the
    // requests of a tick made the solve phase slower (median 9.4 against 8.1
    // ms; a batch waits for its largest member) and the throughput equal, so
    // each request launches its own by default
    p->batch_vcycles = 0;
    return AMG_OK;
}

int amg_server_create(const amg_server_params* p, amg_server** out) {
    return guarded([&] {
        if (!p || !out) throw Error{AMG_EINVAL, "null argument"};
        *out = nullptr;
        if (p->max_slots < 1 || p->setup_threads < 1 || p->setup_threads > 256 || p->maxit < 0)
            throw Error{AMG_EINVAL, "max_slots >= 1, 1 <= setup_threads <= 256 and maxit >= 0"};
        if (p->batch_vcycles != 0 && p->batch_vcycles != 1)
            throw Error{AMG_EINVAL, "batch_vcycles must be 0 or 1"};
        auto S = std::make_unique<amg_server>();
        S->p = *p;
        AMG_CUDA_TRY(cudaGetDevice(&S->device));
        size_t free_b = 0, total_b = 0;
        AMG_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        S->budget = p->hbm_budget_bytes > 0 ? p->hbm_budget_bytes : 0.8 * (double)free_b;
        AMG_CUDA_TRY(cudaStreamCreateWithFlags(&S->batch_stream, cudaStreamNonBlocking));
        AMG_CUDA_TRY(cudaEventCreateWithFlags(&S->batch_ev, cudaEventDisableTiming));
        amg_server* s = S.get();
        s->worker = std::thread(worker_main, s);
        for (int i = 0; i < p->setup_threads; ++i) s->setup_pool.emplace_back(setup_main, s);
        *out = S.release();
    });
}

int amg_submit(amg_server* s, const amg_csr* A, const double* b, double tol, uint64_t* ticket) {
    return guarded([&] {
        if (!s || !A || !b || !ticket) throw Error{AMG_EINVAL, "null argument"};
        if (A->on_device) throw Error{AMG_EINVAL, "amg_submit takes a host matrix"};
        if (A->n <= 0 || A->nnz <= 0 || !A->row_ptr || !A->col || !A->val)
            throw Error{AMG_EINVAL, "empty or null matrix"};
        if (A->row_ptr[0] != 0 || A->row_ptr[A->n] != A->nnz)
            throw Error{AMG_EINVAL, "row_ptr must start at 0 and end at nnz"};
        if (!(tol >= 0.0)) throw Error{AMG_EINVAL, "tol must be >= 0"};
        auto r = std::make_unique<Request>();
        r->n = A->n;
        r->nnz = A->nnz;
        r->rp.assign(A->row_ptr, A->row_ptr + A->n + 1);
        r->ci.assign(A->col, A->col + A->nnz);
        r->va.assign(A->val, A->val + A->nnz);
        r->b.assign(b, b + A->n);
        r->tol = tol;
        r->t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stopping) throw Error{AMG_EINVAL, "the server is stopping"};
            r->ticket = s->next_ticket++;
            *ticket = r->ticket;
            s->queued.push_back(r.get());
            s->reqs.emplace(r->ticket, std::move(r));
            s->n_submitted += 1;
            admit_locked(s);
        }
        s->cv_worker.notify_one();
    });
}

int amg_poll(amg_server* s, uint64_t ticket, double* x_out, amg_solve_info* info,
             amg_request_times* times) {
    if (!s) {
        t_last_error = "null server";
        return AMG_EINVAL;
    }
    std::unique_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) {
            t_last_error = "unknown or already collected ticket";
            return AMG_ENOTFOUND;
        }
        if (it->second->state != Request::kDone) return AMG_PENDING;
        r = std::move(it->second);
        s->reqs.erase(it);
    }
    if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), sizeof(double) * r->n);
    if (info) *info = r->info;
    if (times) {
        const bool admitted = r->t_admit.time_since_epoch().count() != 0;
        const bool ready = r->t_ready.time_since_epoch().count() != 0;
        times->queue_ms = admitted ? ms_between(r->t_submit, r->t_admit) : 0.0;
        times->setup_ms = (admitted && ready) ? ms_between(r->t_admit, r->t_ready) : 0.0;
        times->solve_ms = ready ? ms_between(r->t_ready, r->t_done) : 0.0;
        times->total_ms = ms_between(r->t_submit, r->t_done);
        times->hbm_bytes = r->hbm;
    }
    t_last_error = r->error;
    return r->status;
}

int amg_server_stats_read(amg_server* s, amg_server_stats* out) {
    if (!s || !out) return AMG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->failed = s->n_failed;
    out->queued = (int32_t)s->queued.size();
    out->running = s->admitted;
    out->peak_running = s->peak_running;
    out->hbm_reserved_bytes = s->reserved;
    out->hbm_budget_bytes = s->budget;
    out->batched_vcycles = s->batches;
    out->batched_requests = s->batched_requests;
    return AMG_OK;
}

int amg_server_destroy(amg_server* s) {
    if (!s) return AMG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (Request* r : s->queued) {
            r->status = AMG_EINVAL;
            r->error = "dropped: the server stopped before admitting it";
            r->state = Request::kDone;
        }
        s->queued.clear();
    }
    s->cv_setup.notify_all();
    s->cv_worker.notify_all();
    for (auto& t : s->setup_pool) t.join();
    s->cv_worker.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->batch_stream) {
        cudaStreamSynchronize(s->batch_stream);
        cudaStreamDestroy(s->batch_stream);
    }
    if (s->batch_ev) cudaEventDestroy(s->batch_ev);
    delete s;
    return AMG_OK;
}

}  // extern "C"
