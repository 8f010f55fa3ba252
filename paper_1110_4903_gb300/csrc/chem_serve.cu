// chem_serve.cu -- request server: continuous batching of chemistry steps on
// the device.
//
// Requests from many simulations (each with its own mechanism handle, cell
// count, dt and state buffers) enter one FIFO queue.  A scheduler thread
// admits the head of the queue when its bytes fit in the HBM budget, and
// publishes it to the lane of its (handle, precision): a ring of request
// descriptors in host memory mapped into the device's address space, whose
// cells are numbered consecutively in publication order.  Each lane runs
// persistent instances of the step kernel in its queue mode: a slot that
// frees up inside a running grid claims the next published cell, of
// whichever request comes next, so a request admitted while others run joins
// them inside the same grid (cells of different requests are in flight
// together on every SM).  The kernel counts each request's finished cells;
// the slot that finishes the last one writes the request's completion record
// (with the device timestamps of its first claim and last completion) to
// host memory, which the scheduler polls.
//
// Lanes of different mechanisms share the GPU in space: each kernel
// instance reads a block budget from host memory, blocks beyond it stop
// claiming and leave, and the scheduler gives each lane with work an equal
// share of its full grid, launching and retiring instances as lanes become
// busy or idle.  A warp with no work waits for more (polling the ring every
// 20 us) and leaves when its block is retired or after a bounded linger.
//
// Host states are staged through a device pool of the budget's size on a
// copy stream before publication and copied back after completion.  Each
// request's cells are computed by the same per-cell code as chem_advance_ex
// with the same handle (the work of a cell does not depend on which slot or
// grid runs it), so a result does not depend on what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
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

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

// Ring entries per lane: chunks published and not yet finished at once.
constexpr int kRing = 1024;
// Cells per published chunk: requests are published in chunks, interleaved
// across the lane's active requests (pump), so a request that arrives while a
// large one runs is claimed within one window, not after all of its cells.
// Chunk seq owns the virtual cells from seq * kChunkCells on.
constexpr int64_t kChunkCells = 1LL << kServeChunkLog;
// Kernel instances per lane at once (each with its own block budget).
constexpr int kMaxInstances = 4;
// A warp with no work leaves after this long at most.
constexpr long long kLingerNs = 50LL * 1000 * 1000;
// A lane without requests retires its kernel instances after this long.
constexpr double kIdleRetireS = 2e-3;
// Lanes a server holds at most: their memory and streams are allocated when
// the server is created, because allocating mapped host memory while a
// lane's persistent kernel runs may wait for that kernel.
constexpr int kMaxLanes = 16;
constexpr size_t kLaneHostBytes = sizeof(ServeDesc) * kRing + sizeof(ServeDone) * kRing + 4 * 64;
// device memory of a lane: the chunk being handed out, error, the copies of
// tail, the poll times and the budgets (one per instance) in the first 256
// bytes; per ring entry the cells done, first claim, last completion and the
// claim counter; the descriptor copies
constexpr size_t kLaneDevBytes = 256 + 4 * sizeof(unsigned long long) * kRing + sizeof(ServeDesc) * kRing;
static_assert(192 + kMaxInstances * (sizeof(unsigned long long) + sizeof(int)) <= 256, "lane header");
static_assert((256 + 4 * sizeof(unsigned long long) * kRing) % 64 == 0, "descriptor copies aligned");

enum Phase { kQueued = 0, kStaging = 1, kPublished = 2, kReturning = 3, kFinished = 4 };

struct Req {
    uint64_t ticket = 0;
    chem_request r{};
    int prec = 0;
    size_t bytes = 0;        // bytes counted against the budget
    int state = CHEM_REQ_QUEUED;
    int phase = kQueued;
    int error = CHEM_OK;
    size_t pool_off = 0;
    bool pooled = false;
    int lane = -1;
    long long seq = -1;
    double *d_rho = nullptr, *d_e = nullptr, *d_T = nullptr;   // device buffers the kernel uses
    int32_t *d_st = nullptr;
    cudaEvent_t ev = nullptr;                                   // staging or return copies
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t pos = 0;          // cells published so far
    double t_last_chunk = 0;  // when its last chunk was published
    int chunks_out = 0;       // chunks published and not finished
    unsigned long long dev_t0 = ~0ULL, dev_t1 = 0;
};

struct Instance {
    cudaEvent_t ev = nullptr;
    int cell = -1;           // its block-budget cell
    int grid = 0;
    bool retiring = false;
};

struct Lane {
    Handle *h = nullptr;
    int prec = 0;
    LaunchCfg *cfg = nullptr;
    cudaStream_t streams[kMaxInstances] = {};   // one per block-budget cell: instances run concurrently
    // host memory mapped into the device's address space
    ServeDesc *desc = nullptr;
    ServeDone *fin = nullptr;
    unsigned long long *tail = nullptr;
    unsigned long long *front = nullptr;   // where the hand-out of cells stands, written by the kernel
    int *budgets = nullptr;          // [kMaxInstances]
    ServeDesc *d_desc = nullptr;
    ServeDone *d_fin = nullptr;
    unsigned long long *d_tail = nullptr;
    unsigned long long *d_front = nullptr;
    int *d_budgets = nullptr;
    // device memory: next, error, then done / t_first / t_last per entry
    void *dev = nullptr;
    unsigned long long *chunk = nullptr, *done = nullptr, *t_first = nullptr, *t_last = nullptr;
    unsigned long long *claimed = nullptr;                   // [kRing]
    unsigned long long *dtail = nullptr, *dpoll = nullptr;   // dpoll [kMaxInstances]
    int *dbudget = nullptr;                                  // [kMaxInstances]
    ServeDesc *mdesc = nullptr;                              // [kRing]
    int *error = nullptr;
    long long next_seq = 0;
    unsigned long long published = 0;        // virtual cells of the published chunks
    long long window = 0;                     // published cells kept ahead of the claims
    std::deque<uint64_t> rr;                  // requests with cells still to publish
    std::map<long long, uint64_t> inflight;   // chunk seq -> ticket, published and unfinished
    std::vector<Instance> inst;
    double idle_since = 0;
};

}  // namespace chem

using namespace chem;

struct chem_server_s {
    chem_server_options opts{};
    int device = 0;
    cudaStream_t copy_stream = nullptr;
    char *lane_host = nullptr;         // kMaxLanes x kLaneHostBytes, mapped
    char *lane_host_dev = nullptr;     // its device address
    char *lane_dev = nullptr;          // kMaxLanes x kLaneDevBytes
    cudaStream_t lane_streams[kMaxLanes][kMaxInstances] = {};
    void *pool_mem = nullptr;
    Pool pool;
    size_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // scheduler wake-up
    std::condition_variable cv_done;   // waiters
    std::deque<uint64_t> queue;        // admitted in this order
    std::vector<uint64_t> staging;     // host requests being copied in
    std::vector<uint64_t> waiting;     // device requests waiting for their ready event
    std::vector<uint64_t> returning;   // host requests being copied out
    std::map<uint64_t, Req> reqs;
    std::vector<Lane *> lanes;
    uint64_t next_ticket = 1;
    int active = 0;                    // admitted and not finished
    bool stop = false;
    std::thread thr;
    long long completed = 0, failed = 0;
    std::atomic<long long> launches{0};
};

namespace {

void free_lane(Lane *L) {
    for (auto st : L->streams)
        if (st) cudaStreamSynchronize(st);
    for (auto &in : L->inst)
        if (in.ev) cudaEventDestroy(in.ev);
    delete L;
}

// The lane of (handle, precision), set up on first use in the memory and
// streams the server allocated when it was created (no allocation here).
int get_lane(chem_server_s *S, Handle *h, int prec, int &idx) {
    for (size_t i = 0; i < S->lanes.size(); ++i)
        if (S->lanes[i]->h == h && S->lanes[i]->prec == prec) {
            idx = (int)i;
            return CHEM_OK;
        }
    const int li = (int)S->lanes.size();
    if (li >= kMaxLanes) return fail(CHEM_E_UNSUPPORTED, "more than %d (handle, precision) lanes", kMaxLanes);
    Lane *L = new Lane();
    L->h = h;
    L->prec = prec;
    int rc = get_cfg(h, prec, h->lanes[prec], &L->cfg, true);
    if (rc) {
        delete L;
        return rc;
    }
    for (int c = 0; c < kMaxInstances; ++c) L->streams[c] = S->lane_streams[li][c];
    char *hp = S->lane_host + (size_t)li * kLaneHostBytes;
    char *dp = S->lane_host_dev + (size_t)li * kLaneHostBytes;
    memset(hp, 0, kLaneHostBytes);
    L->desc = reinterpret_cast<ServeDesc *>(hp);
    L->fin = reinterpret_cast<ServeDone *>(hp + sizeof(ServeDesc) * kRing);
    const size_t toff = sizeof(ServeDesc) * kRing + sizeof(ServeDone) * kRing;
    L->tail = reinterpret_cast<unsigned long long *>(hp + toff);
    L->budgets = reinterpret_cast<int *>(hp + toff + 128);
    L->front = reinterpret_cast<unsigned long long *>(hp + toff + 192);
    for (int i = 0; i < kRing; ++i) {
        L->desc[i].seq = -1;
        L->fin[i].seq = -1;
    }
    L->d_desc = reinterpret_cast<ServeDesc *>(dp);
    L->d_fin = reinterpret_cast<ServeDone *>(dp + sizeof(ServeDesc) * kRing);
    L->d_tail = reinterpret_cast<unsigned long long *>(dp + toff);
    L->d_budgets = reinterpret_cast<int *>(dp + toff + 128);
    L->d_front = reinterpret_cast<unsigned long long *>(dp + toff + 192);
    // cells kept published ahead of the claims: a quarter of a grid of
    // slots (what the slots claim in a fraction of a cell's time, far more
    // than one host pass publishes; a request that arrives while a large one
    // runs waits behind no more than that: 1.5 grids measured a small
    // request p50 of 28 ms during a 2^18-cell request, a quarter 18 ms),
    // and never less than the current chunk and one more (the kernels
    // report the current chunk's start, so a window of one chunk would
    // publish nothing beyond it)
    const long long slots = (long long)L->cfg->grid * (L->cfg->block / 32) * (32 / L->cfg->G);
    L->window = std::max<long long>(slots / 4, 2 * kChunkCells);
    char *d = S->lane_dev + (size_t)li * kLaneDevBytes;
    L->chunk = reinterpret_cast<unsigned long long *>(d);
    L->error = reinterpret_cast<int *>(d + 64);
    L->dtail = reinterpret_cast<unsigned long long *>(d + 128);
    L->dpoll = reinterpret_cast<unsigned long long *>(d + 192);
    L->dbudget = reinterpret_cast<int *>(d + 192 + kMaxInstances * sizeof(unsigned long long));
    L->done = reinterpret_cast<unsigned long long *>(d + 256);
    L->t_first = L->done + kRing;
    L->t_last = L->t_first + kRing;
    L->claimed = L->t_last + kRing;
    L->mdesc = reinterpret_cast<ServeDesc *>(L->claimed + kRing);
    // counters on the lane's first stream, ahead of its first kernel there;
    // instances on its other streams wait for them
    cudaError_t ce = cudaMemsetAsync(d, 0, kLaneDevBytes, L->streams[0]);
    if (ce == cudaSuccess)
        ce = cudaMemsetAsync(L->t_first, 0xff, sizeof(unsigned long long) * kRing, L->streams[0]);
    // no descriptor copies yet: every sequence number -1
    if (ce == cudaSuccess) ce = cudaMemsetAsync(L->mdesc, 0xff, sizeof(ServeDesc) * kRing, L->streams[0]);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(L->streams[0]);
    if (ce != cudaSuccess) {
        delete L;
        return cuda_fail(ce, "initialising the lane counters");
    }
    S->lanes.push_back(L);
    idx = li;
    return CHEM_OK;
}

// Launches one kernel instance of the lane with `grid` blocks.
int launch_instance(chem_server_s *S, Lane *L, int grid) {
    int cell = -1;
    for (int c = 0; c < kMaxInstances; ++c) {
        bool used = false;
        for (auto &in : L->inst) used |= in.cell == c;
        if (!used) {
            cell = c;
            break;
        }
    }
    if (cell < 0) return CHEM_OK;   // every budget cell is held: the instances already running stay
    Instance in;
    in.cell = cell;
    in.grid = grid;
    reinterpret_cast<volatile int *>(L->budgets)[cell] = grid;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    cudaError_t ce = cudaEventCreateWithFlags(&in.ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return cuda_fail(ce, "instance event");
    DeviceMech m = L->h->mech;
    StepOptions o = step_options(L->h, L->prec);
    StepBatch b{};
    b.queue.desc = L->d_desc;
    b.queue.fin = L->d_fin;
    b.queue.tail = L->d_tail;
    b.queue.front = L->d_front;
    b.queue.budget = L->d_budgets + cell;
    b.queue.mdesc = L->mdesc;
    b.queue.dtail = L->dtail;
    b.queue.dbudget = L->dbudget + cell;
    b.queue.dpoll = L->dpoll + cell;
    b.queue.chunk = L->chunk;
    b.queue.claimed = L->claimed;
    b.queue.done = L->done;
    b.queue.t_first = L->t_first;
    b.queue.t_last = L->t_last;
    b.queue.cap = kRing;
    b.queue.linger_ns = kLingerNs;
    b.queue.error = L->error;
    void *args[] = {&m, &o, &b};
    cudaStream_t st = L->streams[cell];
    // the instance's budget copy, ahead of it on its stream (the kernel
    // refreshes it from host memory while it runs)
    ce = cudaMemcpyAsync(L->dbudget + cell, L->budgets + cell, sizeof(int), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaLaunchKernel(L->cfg->fn, dim3((unsigned)grid), dim3(L->cfg->block), args, L->cfg->smem, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(in.ev, st);
    if (ce != cudaSuccess) {
        cudaEventDestroy(in.ev);
        return cuda_fail(ce, "launching a server kernel instance");
    }
    L->inst.push_back(in);
    S->launches.fetch_add(1);
    L->h->launches.fetch_add(1);
    return CHEM_OK;
}

// Writes cells [q.pos, q.pos + c) of a request into its lane's ring as one
// chunk and moves the tail over them.
void publish_chunk(Lane *L, Req &q, int64_t c) {
    const long long seq = L->next_seq++;
    const int e = (int)(seq % kRing);
    volatile ServeDesc *d = L->desc + e;
    const int64_t p = q.pos;
    d->start = seq << kServeChunkLog;
    d->n_cells = c;
    d->ld = q.r.host ? q.r.n_cells : (q.r.ld ? q.r.ld : q.r.n_cells);
    d->rho = q.d_rho + p;
    d->e = q.d_e + p;
    d->T_out = q.d_T ? q.d_T + p : nullptr;
    d->status = q.d_st ? q.d_st + p : nullptr;
    d->dt = q.r.dt;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    d->seq = seq;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    // the chunk's real cells become claimable; its unused numbers up to the
    // next chunk's start are skipped by the claims
    L->published = (unsigned long long)(seq + 1) << kServeChunkLog;
    *reinterpret_cast<volatile unsigned long long *>(L->tail) = ((unsigned long long)seq << kServeChunkLog) + c;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    q.pos += c;
    q.chunks_out++;
    L->inflight[seq] = q.ticket;
}

// Publishes chunks of the lane's active requests while fewer than `window`
// virtual cells are published from the chunk the kernels are handing out
// (`front`): next the request with the fewest cells
// left to publish (the shortest first, which keeps the latency of small
// requests low while a large one runs), unless one has had no chunk
// published for kStarveS, which then goes first.
constexpr double kStarveS = 0.05;
void pump(chem_server_s *S, Lane *L) {
    const unsigned long long front = *reinterpret_cast<volatile unsigned long long *>(L->front);
    const double now = now_s();
    while (!L->rr.empty() && (long long)(L->published - std::min(front, L->published)) < L->window &&
           (long long)L->inflight.size() < kRing - 1) {
        auto pick = L->rr.begin();
        int64_t best = INT64_MAX;
        for (auto it = L->rr.begin(); it != L->rr.end(); ++it) {
            const Req &q = S->reqs[*it];
            if (now - q.t_last_chunk > kStarveS) {
                pick = it;
                break;
            }
            const int64_t left = q.r.n_cells - q.pos;
            if (left < best) {
                best = left;
                pick = it;
            }
        }
        const uint64_t t = *pick;
        L->rr.erase(pick);
        Req &q = S->reqs[t];
        publish_chunk(L, q, std::min<int64_t>(kChunkCells, q.r.n_cells - q.pos));
        q.t_last_chunk = now;
        if (q.pos < q.r.n_cells) L->rr.push_back(t);
    }
}

// A request ready for the device joins its lane's requests to publish.
void publish(chem_server_s *S, Req &q) {
    Lane *L = S->lanes[q.lane];
    q.phase = kPublished;
    q.state = CHEM_REQ_RUNNING;
    q.t_start = now_s();
    q.pos = 0;
    q.t_last_chunk = q.t_start;
    L->rr.push_back(q.ticket);
    L->idle_since = 0;
    pump(S, L);
}

void finish(chem_server_s *S, Req &q, int state, int error) {
    q.state = state;
    q.error = error;
    q.phase = kFinished;
    q.t_done = now_s();
    if (q.pooled) S->pool.release(q.pool_off, q.bytes);
    q.pooled = false;
    S->in_use -= q.bytes;
    S->active--;
    if (q.ev) {
        cudaEventDestroy(q.ev);
        q.ev = nullptr;
    }
    if (state == CHEM_REQ_DONE)
        S->completed++;
    else
        S->failed++;
    S->cv_done.notify_all();
}

// Completion records of the lanes' published requests.
bool poll_lanes(chem_server_s *S) {
    bool any = false;
    for (Lane *L : S->lanes) {
        for (auto it = L->inflight.begin(); it != L->inflight.end();) {
            const long long seq = it->first;
            volatile ServeDone *f = L->fin + (seq % kRing);
            if (f->seq != seq) {
                ++it;
                continue;
            }
            std::atomic_thread_fence(std::memory_order_acquire);
            Req &q = S->reqs[it->second];
            const unsigned long long tf = f->t_first, tl = f->t_last;
            q.dev_t0 = std::min(q.dev_t0, tf);
            q.dev_t1 = std::max(q.dev_t1, tl);
            q.chunks_out--;
            it = L->inflight.erase(it);
            any = true;
            if (q.pos < q.r.n_cells || q.chunks_out > 0) continue;   // more chunks to come
            if (q.r.host) {
                // copy the results back to the caller's host buffers
                const chem_request &r = q.r;
                const int ns = L->h->ns;
                const int64_t n = r.n_cells, ld = r.ld ? r.ld : r.n_cells;
                cudaError_t ce = cudaMemcpy2DAsync(r.rho_s, (size_t)ld * 8, q.d_rho, (size_t)n * 8, (size_t)n * 8, ns,
                                                   cudaMemcpyDeviceToHost, S->copy_stream);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(r.e, q.d_e, (size_t)n * 8, cudaMemcpyDeviceToHost, S->copy_stream);
                if (ce == cudaSuccess && r.T_out)
                    ce = cudaMemcpyAsync(r.T_out, q.d_T, (size_t)n * 8, cudaMemcpyDeviceToHost, S->copy_stream);
                if (ce == cudaSuccess && r.status)
                    ce = cudaMemcpyAsync(r.status, q.d_st, (size_t)n * 4, cudaMemcpyDeviceToHost, S->copy_stream);
                if (ce == cudaSuccess) ce = cudaEventRecord(q.ev, S->copy_stream);
                if (ce != cudaSuccess) {
                    finish(S, q, CHEM_REQ_FAILED, cuda_fail(ce, "returning a request"));
                } else {
                    q.phase = kReturning;
                    S->returning.push_back(q.ticket);
                }
            } else {
                finish(S, q, CHEM_REQ_DONE, CHEM_OK);
            }
        }
        pump(S, L);
    }
    return any;
}

// Instances: reap finished ones; give each lane with work an equal share of
// its full grid; retire the instances of lanes idle for a while.
void manage_instances(chem_server_s *S) {
    int active_lanes = 0;
    for (Lane *L : S->lanes) active_lanes += !L->inflight.empty() || !L->rr.empty();
    const double now = now_s();
    for (Lane *L : S->lanes) {
        for (auto it = L->inst.begin(); it != L->inst.end();) {
            if (cudaEventQuery(it->ev) == cudaSuccess) {
                cudaEventDestroy(it->ev);
                it = L->inst.erase(it);
            } else {
                ++it;
            }
        }
        volatile int *bud = L->budgets;
        if (L->inflight.empty() && L->rr.empty()) {
            if (L->idle_since == 0) L->idle_since = now;
            if (S->stop || now - L->idle_since > kIdleRetireS)
                for (auto &in : L->inst)
                    if (!in.retiring) {
                        in.retiring = true;
                        bud[in.cell] = 0;
                    }
            continue;
        }
        const int full = L->cfg->grid;
        const int want = std::max(1, (full + active_lanes - 1) / active_lanes);
        // the share, handed to the live instances in launch order; an extra
        // instance covers a shortfall (its blocks take the SMs other lanes'
        // retiring blocks free)
        int given = 0;
        for (auto &in : L->inst) {
            if (in.retiring) continue;
            const int b = std::max(0, std::min(in.grid, want - given));
            if (bud[in.cell] != b) bud[in.cell] = b;
            // blocks past a lowered budget leave for good: the instance only shrinks
            in.grid = b;
            in.retiring = b == 0;
            given += b;
        }
        if (want - given >= std::min(8, want)) launch_instance(S, L, want - given);
    }
    std::atomic_thread_fence(std::memory_order_seq_cst);
}

// Admits the head of the queue while the budget and the rings allow.
void admit(chem_server_s *S) {
    while (!S->queue.empty()) {
        Req &q = S->reqs[S->queue.front()];
        if (q.state == CHEM_REQ_CANCELLED) {
            S->queue.pop_front();
            continue;
        }
        if (S->active >= S->opts.max_inflight || S->in_use + q.bytes > S->budget) break;
        int li = -1;
        int rc = get_lane(S, q.r.mech, q.prec, li);
        if (rc) {
            S->queue.pop_front();
            S->in_use += q.bytes;
            S->active++;
            finish(S, q, CHEM_REQ_FAILED, rc);
            continue;
        }
        Lane *L = S->lanes[li];
        if (q.r.host && !S->pool.alloc(q.bytes, q.pool_off)) break;   // fragmented: wait
        S->queue.pop_front();
        q.pooled = q.r.host;
        S->in_use += q.bytes;
        S->active++;
        q.lane = li;
        q.state = CHEM_REQ_RUNNING;
        q.t_start = now_s();
        const chem_request &r = q.r;
        if (!r.host) {
            q.d_rho = r.rho_s;
            q.d_e = r.e;
            q.d_T = r.T_out;
            q.d_st = r.status;
            if (r.ready_event) {
                q.phase = kStaging;
                S->waiting.push_back(q.ticket);
            } else {
                publish(S, q);
            }
            continue;
        }
        const int ns = q.r.mech->ns;
        const int64_t n = r.n_cells, ld = r.ld ? r.ld : r.n_cells;
        char *base = static_cast<char *>(S->pool_mem) + q.pool_off;
        q.d_rho = reinterpret_cast<double *>(base);
        q.d_e = q.d_rho + (size_t)n * ns;
        double *d_T = q.d_e + n;
        int32_t *d_st = reinterpret_cast<int32_t *>(d_T + n);
        q.d_T = r.T_out ? d_T : nullptr;
        q.d_st = r.status ? d_st : nullptr;
        cudaError_t ce = cudaEventCreateWithFlags(&q.ev, cudaEventDisableTiming);
        if (ce == cudaSuccess)
            ce = cudaMemcpy2DAsync(q.d_rho, (size_t)n * 8, r.rho_s, (size_t)ld * 8, (size_t)n * 8, ns,
                                   cudaMemcpyHostToDevice, S->copy_stream);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(q.d_e, r.e, (size_t)n * 8, cudaMemcpyHostToDevice, S->copy_stream);
        if (ce == cudaSuccess) ce = cudaEventRecord(q.ev, S->copy_stream);
        if (ce != cudaSuccess) {
            finish(S, q, CHEM_REQ_FAILED, cuda_fail(ce, "staging a request"));
            continue;
        }
        q.phase = kStaging;
        S->staging.push_back(q.ticket);
    }
}

// Staged host requests and device requests whose ready event has fired are
// published; returned host requests are done.
void progress_copies(chem_server_s *S) {
    for (auto it = S->staging.begin(); it != S->staging.end();) {
        Req &q = S->reqs[*it];
        const cudaError_t e = cudaEventQuery(q.ev);
        if (e == cudaErrorNotReady) {
            ++it;
            continue;
        }
        it = S->staging.erase(it);
        if (e != cudaSuccess)
            finish(S, q, CHEM_REQ_FAILED, cuda_fail(e, "staging a request"));
        else
            publish(S, q);
    }
    for (auto it = S->waiting.begin(); it != S->waiting.end();) {
        Req &q = S->reqs[*it];
        const cudaError_t e = cudaEventQuery((cudaEvent_t)q.r.ready_event);
        if (e == cudaErrorNotReady) {
            ++it;
            continue;
        }
        it = S->waiting.erase(it);
        if (e != cudaSuccess)
            finish(S, q, CHEM_REQ_FAILED, cuda_fail(e, "the request's ready event"));
        else
            publish(S, q);
    }
    for (auto it = S->returning.begin(); it != S->returning.end();) {
        Req &q = S->reqs[*it];
        const cudaError_t e = cudaEventQuery(q.ev);
        if (e == cudaErrorNotReady) {
            ++it;
            continue;
        }
        it = S->returning.erase(it);
        finish(S, q, e == cudaSuccess ? CHEM_REQ_DONE : CHEM_REQ_FAILED,
               e == cudaSuccess ? CHEM_OK : cuda_fail(e, "returning a request"));
    }
}

void scheduler(chem_server_s *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        poll_lanes(S);
        progress_copies(S);
        admit(S);
        manage_instances(S);
        bool instances = false;
        for (Lane *L : S->lanes) instances |= !L->inst.empty();
        if (S->stop && S->active == 0 && !instances) break;
        if (S->active > 0 || instances)
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
    o->max_inflight = 64;
    o->queue_capacity = 100000;
    return CHEM_OK;
}

int chem_server_create(const chem_server_options *opts, chem_server_t *out) {
    if (!out) return fail(CHEM_E_INVALID_ARG, "output pointer is NULL");
    *out = nullptr;
    chem_server_options o;
    chem_server_default_options(&o);
    if (opts) o = *opts;
    if (o.max_inflight < 1 || o.max_inflight > kRing - 1) return fail(CHEM_E_INVALID_ARG, "max_inflight %d", o.max_inflight);
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
    ce = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaHostAlloc((void **)&S->lane_host, kLaneHostBytes * kMaxLanes, cudaHostAllocMapped);
    if (ce == cudaSuccess) ce = cudaHostGetDevicePointer((void **)&S->lane_host_dev, S->lane_host, 0);
    if (ce == cudaSuccess) ce = cudaMalloc(&S->lane_dev, kLaneDevBytes * kMaxLanes);
    for (int l = 0; l < kMaxLanes && ce == cudaSuccess; ++l)
        for (int c = 0; c < kMaxInstances && ce == cudaSuccess; ++c)
            ce = cudaStreamCreateWithFlags(&S->lane_streams[l][c], cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        for (auto &row : S->lane_streams)
            for (auto st : row)
                if (st) cudaStreamDestroy(st);
        if (S->lane_dev) cudaFree(S->lane_dev);
        if (S->lane_host) cudaFreeHost(S->lane_host);
        if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
        cudaFree(S->pool_mem);
        delete S;
        return cuda_fail(ce, "request-server setup");
    }
    S->thr = std::thread(scheduler, S);
    *out = S;
    return CHEM_OK;
}

int chem_server_destroy(chem_server_t S) {
    if (!S) return fail(CHEM_E_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        // queued requests are cancelled; admitted ones finish
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
    S->cv_done.notify_all();
    S->thr.join();
    cudaStreamSynchronize(S->copy_stream);
    for (Lane *L : S->lanes) free_lane(L);
    for (auto &kv : S->reqs)
        if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    for (auto &row : S->lane_streams)
        for (auto st : row)
            if (st) cudaStreamDestroy(st);
    cudaFree(S->lane_dev);
    cudaFreeHost(S->lane_host);
    cudaStreamDestroy(S->copy_stream);
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
    out->dev_first_ns = q.dev_t0 == ~0ULL ? 0 : q.dev_t0;
    out->dev_last_ns = q.state == CHEM_REQ_DONE ? q.dev_t1 : 0;
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
    out->running = S->active;
    out->completed = S->completed;
    out->failed = S->failed;
    out->bytes_in_use = (int64_t)S->in_use;
    out->budget_bytes = (int64_t)S->budget;
    out->launches = S->launches.load();
    int64_t inst = 0;
    for (Lane *L : S->lanes) inst += (int64_t)L->inst.size();
    out->kernel_instances = inst;
    int err = 0;
    for (Lane *L : S->lanes) {
        int e = 0;
        if (cudaMemcpy(&e, L->error, sizeof e, cudaMemcpyDeviceToHost) == cudaSuccess) err |= e;
    }
    out->queue_errors = err;
    return CHEM_OK;
}

}  // extern "C"
