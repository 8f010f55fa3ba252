// chem_serve.cu -- request server: continuous batching of chemistry steps.
//
// Requests from many simulations (each its own mechanism handle, cell count,
// dt and state buffers) go into one FIFO queue.  A scheduler thread admits
// the head of the queue as soon as a stream slot is free and the request's
// bytes fit in the HBM budget, launches it on that slot's stream, and
// retires it when the slot's event completes; requests admitted while
// others run overlap with them on the device.  States that live on the
// device are stepped in place; host states are staged through a device pool
// of exactly the budget size.  Each request is computed by the same kernel
// on the same per-cell arithmetic whether it runs alone or in a mix, so its
// result does not depend on what else is in flight.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/chem.h"
#include "chem_handle.h"

namespace chem {

void destroy_serving(Handle *h) { (void)h; }

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device allocation (offsets only; host side).
class Pool {
  public:
    void init(size_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
        size_ = bytes;
    }
    bool alloc(size_t bytes, size_t &off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

struct Req {
    uint64_t ticket = 0;
    chem_request r{};
    int prec = 0;
    size_t bytes = 0;        // bytes counted against the budget
    int state = CHEM_REQ_QUEUED;
    int error = CHEM_OK;
    int slot = -1;
    size_t pool_off = 0;
    bool pooled = false;
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t ticket = 0;     // 0 = free
};

}  // namespace chem

using namespace chem;

struct chem_server_s {
    chem_server_options opts{};
    int device = 0;
    std::vector<Slot> slots;
    void *pool_mem = nullptr;
    Pool pool;
    size_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // scheduler wake-up
    std::condition_variable cv_done;   // waiters
    std::deque<uint64_t> queue;
    std::map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread thr;
    long long completed = 0, failed = 0;
    std::atomic<long long> launches{0};
};

namespace {

// Launch one admitted request on its slot (called with the lock held).
int launch_request(chem_server_s *S, Req &q) {
    Slot &sl = S->slots[q.slot];
    Handle *h = q.r.mech;
    const chem_request &r = q.r;
    const int ns = h->ns;
    const int64_t n = r.n_cells, ld = r.ld ? r.ld : r.n_cells;
    double *rho = r.rho_s, *e = r.e, *T_out = r.T_out;
    int32_t *status = r.status;
    double *d_T = nullptr;
    int32_t *d_st = nullptr;
    cudaError_t ce = cudaSuccess;
    if (r.ready_event) {
        ce = cudaStreamWaitEvent(sl.stream, (cudaEvent_t)r.ready_event, 0);
        if (ce != cudaSuccess) return cuda_fail(ce, "waiting for the request's ready event");
    }
    if (r.host) {
        char *base = static_cast<char *>(S->pool_mem) + q.pool_off;
        double *d_rho = reinterpret_cast<double *>(base);
        double *d_e = d_rho + (size_t)n * ns;
        d_T = d_e + n;
        d_st = reinterpret_cast<int32_t *>(d_T + n);
        ce = cudaMemcpy2DAsync(d_rho, (size_t)n * 8, rho, (size_t)ld * 8, (size_t)n * 8, ns,
                               cudaMemcpyHostToDevice, sl.stream);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_e, e, (size_t)n * 8, cudaMemcpyHostToDevice, sl.stream);
        if (ce != cudaSuccess) return cuda_fail(ce, "staging a request");
        rho = d_rho;
        e = d_e;
    }
    chem_advance_args a;
    memset(&a, 0, sizeof a);
    a.n_cells = n;
    a.ld = r.host ? n : ld;
    a.rho_s = rho;
    a.e = e;
    a.dt = r.dt;
    a.T_out = r.host ? (T_out ? d_T : nullptr) : T_out;
    a.status = r.host ? (status ? d_st : nullptr) : status;
    a.stream = sl.stream;
    a.precision = q.prec;
    int rc = chem_advance_ex(h, &a);
    if (rc) return rc;
    S->launches.fetch_add(1);
    if (r.host) {
        ce = cudaMemcpy2DAsync(r.rho_s, (size_t)ld * 8, rho, (size_t)n * 8, (size_t)n * 8, ns,
                               cudaMemcpyDeviceToHost, sl.stream);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(r.e, e, (size_t)n * 8, cudaMemcpyDeviceToHost, sl.stream);
        if (ce == cudaSuccess && T_out)
            ce = cudaMemcpyAsync(T_out, d_T, (size_t)n * 8, cudaMemcpyDeviceToHost, sl.stream);
        if (ce == cudaSuccess && status)
            ce = cudaMemcpyAsync(status, d_st, (size_t)n * 4, cudaMemcpyDeviceToHost, sl.stream);
        if (ce != cudaSuccess) return cuda_fail(ce, "returning a request");
    }
    ce = cudaEventRecord(sl.done, sl.stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "recording the completion event");
    return CHEM_OK;
}

void release_request(chem_server_s *S, Req &q) {
    if (q.pooled) S->pool.release(q.pool_off, q.bytes);
    q.pooled = false;
    S->in_use -= q.bytes;
    if (q.slot >= 0) S->slots[q.slot].ticket = 0;
    q.slot = -1;
}

void scheduler(chem_server_s *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // retire finished requests
        bool inflight = false;
        for (auto &sl : S->slots) {
            if (!sl.ticket) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                inflight = true;
                continue;
            }
            Req &r = S->reqs[sl.ticket];
            r.t_done = now_s();
            if (q == cudaSuccess) {
                r.state = CHEM_REQ_DONE;
                S->completed++;
            } else {
                r.state = CHEM_REQ_FAILED;
                r.error = CHEM_E_CUDA;
                S->failed++;
            }
            release_request(S, r);
            S->cv_done.notify_all();
        }
        // admit from the head of the queue while slots and budget allow
        while (!S->queue.empty()) {
            Req &q = S->reqs[S->queue.front()];
            if (q.state == CHEM_REQ_CANCELLED) {
                S->queue.pop_front();
                continue;
            }
            int free_slot = -1;
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].ticket) {
                    free_slot = (int)i;
                    break;
                }
            if (free_slot < 0 || S->in_use + q.bytes > S->budget) break;
            if (q.r.host) {
                if (!S->pool.alloc(q.bytes, q.pool_off)) break;   // fragmented: wait
                q.pooled = true;
            }
            S->queue.pop_front();
            S->in_use += q.bytes;
            q.slot = free_slot;
            S->slots[free_slot].ticket = q.ticket;
            q.t_start = now_s();
            q.state = CHEM_REQ_RUNNING;
            const int rc = launch_request(S, q);
            if (rc) {
                q.state = CHEM_REQ_FAILED;
                q.error = rc;
                q.t_done = now_s();
                S->failed++;
                // the slot's stream may hold staged copies; wait for them
                cudaStreamSynchronize(S->slots[free_slot].stream);
                release_request(S, q);
                S->cv_done.notify_all();
            } else {
                inflight = true;
            }
        }
        if (S->stop && !inflight) break;
        if (inflight)
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    }
}

}  // namespace

extern "C" {

int chem_server_default_options(chem_server_options *o) {
    if (!o) return fail(CHEM_E_INVALID_ARG, "options pointer is NULL");
    o->hbm_budget_bytes = 0;
    o->max_inflight = 8;
    o->queue_capacity = 100000;
    return CHEM_OK;
}

int chem_server_create(const chem_server_options *opts, chem_server_t *out) {
    if (!out) return fail(CHEM_E_INVALID_ARG, "output pointer is NULL");
    *out = nullptr;
    chem_server_options o;
    chem_server_default_options(&o);
    if (opts) o = *opts;
    if (o.max_inflight < 1 || o.max_inflight > 64) return fail(CHEM_E_INVALID_ARG, "max_inflight %d", o.max_inflight);
    if (o.queue_capacity < 1) return fail(CHEM_E_INVALID_ARG, "queue_capacity %d", o.queue_capacity);
    if (o.hbm_budget_bytes < 0) return fail(CHEM_E_INVALID_ARG, "hbm_budget_bytes");
    chem_server_s *S = new chem_server_s();
    S->opts = o;
    cudaError_t ce = cudaGetDevice(&S->device);
    if (ce != cudaSuccess) { delete S; return cuda_fail(ce, "cudaGetDevice"); }
    size_t free_b = 0, total_b = 0;
    ce = cudaMemGetInfo(&free_b, &total_b);
    if (ce != cudaSuccess) { delete S; return cuda_fail(ce, "cudaMemGetInfo"); }
    S->budget = o.hbm_budget_bytes ? (size_t)o.hbm_budget_bytes : free_b / 4;
    if (S->budget > free_b) { delete S; return fail(CHEM_E_OOM, "budget %zu > free %zu", S->budget, free_b); }
    ce = cudaMalloc(&S->pool_mem, S->budget);
    if (ce != cudaSuccess) { delete S; return fail(CHEM_E_OOM, "server pool (%zu bytes)", S->budget); }
    S->pool.init(S->budget);
    S->slots.resize(o.max_inflight);
    for (auto &sl : S->slots) {
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    S->thr = std::thread(scheduler, S);
    *out = S;
    return CHEM_OK;
}

int chem_server_destroy(chem_server_t S) {
    if (!S) return fail(CHEM_E_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        // queued requests are cancelled; running ones finish
        for (uint64_t t : S->queue) {
            Req &r = S->reqs[t];
            if (r.state == CHEM_REQ_QUEUED) {
                r.state = CHEM_REQ_CANCELLED;
                r.t_done = now_s();
            }
        }
        S->queue.clear();
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->thr.join();
    for (auto &sl : S->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaEventDestroy(sl.done);
        cudaStreamDestroy(sl.stream);
    }
    cudaFree(S->pool_mem);
    delete S;
    return CHEM_OK;
}

int chem_submit(chem_server_t S, const chem_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    if (!r->mech || !r->rho_s || !r->e || r->n_cells < 1 || (r->ld != 0 && r->ld < r->n_cells) ||
        !(r->dt >= 0) || r->dt != r->dt)
        return fail(CHEM_E_INVALID_ARG, "bad request");
    Handle *h = r->mech;
    const int prec = r->precision < 0 ? h->opts.precision : r->precision;
    if (prec != CHEM_FP64 && prec != CHEM_MIXED) return fail(CHEM_E_INVALID_ARG, "precision %d", prec);
    if (h->device != S->device) return fail(CHEM_E_INVALID_ARG, "handle and server on different devices");
    Req q;
    q.r = *r;
    q.prec = prec;
    q.bytes = (size_t)r->n_cells * ((size_t)h->ns * 8 + 8 + 8 + 4) + 1024;
    if (q.bytes > S->budget)
        return fail(CHEM_E_OVER_BUDGET, "request of %zu bytes exceeds the budget of %zu", q.bytes, S->budget);
    q.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(CHEM_E_INVALID_ARG, "server is shutting down");
        if ((long long)S->queue.size() >= S->opts.queue_capacity)
            return fail(CHEM_E_OVER_BUDGET, "queue full (%d)", S->opts.queue_capacity);
        q.ticket = S->next_ticket++;
        *ticket = q.ticket;
        S->reqs[q.ticket] = q;
        S->queue.push_back(q.ticket);
    }
    S->cv_work.notify_one();
    return CHEM_OK;
}

static void fill_result(const Req &q, chem_result *out) {
    out->state = q.state;
    out->error = q.error;
    out->t_submit = q.t_submit;
    out->t_start = q.t_start;
    out->t_done = q.t_done;
}

int chem_poll(chem_server_t S, uint64_t ticket, chem_result *out) {
    if (!S || !out) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CHEM_E_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
    fill_result(it->second, out);
    return CHEM_OK;
}

int chem_wait(chem_server_t S, uint64_t ticket, int64_t timeout_us, chem_result *out) {
    if (!S || !out) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CHEM_E_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
    auto finished = [&] {
        const int st = S->reqs[ticket].state;
        return st == CHEM_REQ_DONE || st == CHEM_REQ_FAILED || st == CHEM_REQ_CANCELLED;
    };
    if (timeout_us < 0) {
        S->cv_done.wait(lk, finished);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished)) {
        fill_result(S->reqs[ticket], out);
        return fail(CHEM_E_TIMEOUT, "ticket %llu not finished after %lld us", (unsigned long long)ticket,
                    (long long)timeout_us);
    }
    fill_result(S->reqs[ticket], out);
    return CHEM_OK;
}

int chem_cancel(chem_server_t S, uint64_t ticket) {
    if (!S) return fail(CHEM_E_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CHEM_E_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
    if (it->second.state != CHEM_REQ_QUEUED)
        return fail(CHEM_E_INVALID_ARG, "ticket %llu is no longer queued", (unsigned long long)ticket);
    it->second.state = CHEM_REQ_CANCELLED;
    it->second.t_done = now_s();
    S->cv_done.notify_all();
    return CHEM_OK;
}

int chem_release(chem_server_t S, uint64_t ticket) {
    if (!S) return fail(CHEM_E_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CHEM_E_NOT_FOUND, "ticket %llu", (unsigned long long)ticket);
    const int st = it->second.state;
    if (st == CHEM_REQ_QUEUED || st == CHEM_REQ_RUNNING)
        return fail(CHEM_E_INVALID_ARG, "ticket %llu has not finished", (unsigned long long)ticket);
    S->reqs.erase(it);
    return CHEM_OK;
}

int chem_server_stats(chem_server_t S, chem_server_stats_t *out) {
    if (!S || !out) return fail(CHEM_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int64_t)S->queue.size();
    int64_t run = 0;
    for (auto &sl : S->slots) run += sl.ticket != 0;
    out->running = run;
    out->completed = S->completed;
    out->failed = S->failed;
    out->bytes_in_use = (int64_t)S->in_use;
    out->budget_bytes = (int64_t)S->budget;
    out->launches = S->launches.load();
    return CHEM_OK;
}

}  // extern "C"
