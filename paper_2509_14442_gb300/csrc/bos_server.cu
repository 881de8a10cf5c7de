// Request server: continuous batching of forward and forward+adjoint renders on one GPU.
//
// Requests arrive at any time (bos_submit, from any thread) and queue FIFO.  A scheduler
// thread admits the queue head as soon as (a) fewer than `slots` requests are in flight
// and (b) the request's exact device footprint fits in the free space of the server's
// arena, a single device allocation of mem_limit_bytes made once at creation (first-fit
// with coalescing; nothing is allocated or freed per request).
//
// Admitted requests are executed by batched launches.  The field build of a request is
// enqueued at admission; after it, the request's warp tiles join a shared pool, and each
// batched launch (render_batch_kernel, adjoint_batch_kernel) pulls warp tiles of admitted
// requests in its phase from one device work list, oldest request first, up to a bounded
// amount of work per launch, so a request that arrives while others run joins the next
// launch.  Render launches (with L_BOS) run on one stream, adjoint launches (with the
// gradient epilogues) on another and field builds on a third, so they overlap on the
// device and fill each other's tails; a request's hand-overs from its build to its render
// launches and from its render phase to its adjoint are events.  An event behind its last kernel marks completion.  Launches are cut at batch boundaries rather than kept resident: the
// gathers read the field stores through the non-coherent L1 path, which may assume the
// data does not change while a kernel runs, and stores are rebuilt in recycled arena
// memory as requests come and go.  Requests of other kinds (float64 or plain float32
// stores, RK4, the refracted projector connection) run their own launches on the render
// stream, in admission order.  No kernel waits on the host or on another kernel:
// the only waits are host-side and bounded (bos_wait, bos_server_destroy).
//
// The fake executor (BOS_SERVER_FAKE_EXECUTOR) runs the same admission, slot and memory
// logic without any CUDA call: an admitted request "runs" for a time proportional to
// its footprint.  It exists to test the scheduler on machines without a GPU.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/bos.h"
#include "bos_ctx_internal.h"
#include "bos_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing of neighbouring free ranges.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = 0;
    }
    bool alloc(size_t n, size_t* off) {
        n = bos::align_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = bos::align_up(n);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
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
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

// Phases of an admitted request on the GPU.
enum Phase { PH_RENDER = 0, PH_ADJOINT = 1, PH_FINISH = 2 };

struct Req {
    bos_request r;
    uint64_t footprint = 0;
    uint64_t t_submit = 0, t_admit = 0, t_done = 0;
    int status = BOS_OK;
    int slot = -1;
    bool done = false;
    size_t off = 0;
    // GPU engine
    uint64_t order = 0;             // admission order
    bool batched = false;
    int phase = PH_FINISH;
    int mode = 0, integ = 0;
    bos::BatchJob J{};
    int tiles[2] = {0, 0}, next[2] = {0, 0};
    double cost = 1.0;              // ray-step bound of one warp tile
    float* dLdI = nullptr;
    cudaEvent_t ev = nullptr;       // behind the request's last kernel
    cudaEvent_t ev_hand = nullptr;  // behind its render phase and L_BOS (forward + adjoint)
    bool handed = false;            // its first adjoint launch waits on ev_hand
    cudaEvent_t ev_build = nullptr; // behind its field build (on the build stream)
    bool built = false;             // its first render launch waits on ev_build
};

struct Slot {
    bos_ctx* ctx = nullptr;
    cudaEvent_t ev = nullptr;       // completion of the slot's request
    cudaEvent_t ev_hand = nullptr;  // its render phase (and L_BOS) done: the adjoint may start
    cudaEvent_t ev_build = nullptr; // its field build done: its render tiles may start
    bool busy = false;
    uint64_t ticket = 0;
    std::atomic<bool> finished{false};
    std::atomic<uint64_t> t_finished{0};
    uint64_t fake_due = 0;
    struct bos_server* owner = nullptr;
};

// One batched launch in flight: its job list (pinned host copy and device copy), work
// counter and completion event.
struct Batch {
    bos::BatchJob* host = nullptr;
    bos::BatchJob* dev = nullptr;
    int* counter = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int phase = 0;
};

constexpr int kMaxBatchJobs = 64;       // jobs per batched launch (= the slot limit)
constexpr int kBatches = 8;             // job-list buffers
constexpr int kInFlight = 2;            // batched launches per phase enqueued ahead of the GPU
// Work per batched launch, in ray-step bounds (a ray's step budget, ~1.6x its actual steps):
// ~10 ms of the GPU, long enough that the tail of a launch (its last warps finishing) is a
// small part of it, short enough that a new request joins soon.
constexpr double kRenderBudget = 1.0e9;
constexpr double kAdjointBudget = 2.5e8;
constexpr int kSegK = 64;               // segment slices of the batched Sharma adjoint hold up to 64 steps

size_t scratch_bytes(const bos_request& r) {   // dL/dI between the loss and the backward
    return r.target_dev ? bos::align_up((size_t)r.cam.width * r.cam.height * sizeof(float)) : 0;
}

}  // namespace

struct bos_server {
    int device = 0;
    int flags = 0;
    uint64_t limit = 0;
    char* base = nullptr;
    Arena arena;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv;        // scheduler wake-ups and waiters
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread sched;
    size_t peak_used = 0;
    // GPU engine: stream 0 carries field builds, render launches and L_BOS; stream 1 the
    // adjoint launches and gradient epilogues, so that the two kinds of launch overlap
    cudaStream_t stream = nullptr, stream_adj = nullptr;
    cudaStream_t stream_build = nullptr;   // field builds of batched requests, overlapping the launches
    Batch batches[kBatches];
    float* seg = nullptr;              // segment slices of the batched Sharma adjoint (in the arena)
    int num_sms = 1;
    uint64_t admitted = 0;
    std::vector<uint64_t> active;      // tickets of admitted, unfinished requests in admission order
    uint64_t n_batches = 0, n_batch_tiles = 0, n_batch_jobs = 0;
    int max_batch_jobs = 0;

    bool fake() const { return flags & BOS_SERVER_FAKE_EXECUTOR; }
    void run();
    void launch(Req& q, Slot& s);
    void finish(Slot& s);
    bool launch_batch(int phase);
    void after_phase(Req& q);
    void fail_request(Req& q, bos_status_t e);
};

namespace {

bos_status_t validate_request(const bos_request* r) {
    if (!r || !r->T_dev || !r->pattern_dev || !r->I_dev) return BOS_ERR_INVALID_ARG;
    if (r->target_dev && (!r->loss_dev || !r->dLdT_dev)) return BOS_ERR_INVALID_ARG;
    // the checks of bos_set_grid / bos_set_geometry, at submission rather than at launch
    bos_status_t e = bos::check_grid_desc(&r->grid, "bos_submit");
    if (e == BOS_OK) e = bos::check_geometry_desc(&r->cam, &r->wall, &r->light, r->pattern_dev, &r->integ, "bos_submit");
    return e;
}

}  // namespace

// A request whose launch failed: let the work already enqueued drain before its memory is
// reused, then mark it finished.
void bos_server::fail_request(Req& q, bos_status_t e) {
    q.status = e;
    q.phase = PH_FINISH;
    q.batched = false;
    cudaStreamSynchronize(stream);
    cudaStreamSynchronize(stream_adj);
    cudaStreamSynchronize(stream_build);
    cudaEventRecord(q.ev, stream);
}

void bos_server::launch(Req& q, Slot& s) {
    if (fake()) {
        // simulated run time: 1 ms + 1 ms per 64 MiB of footprint
        s.fake_due = now_ns() + 1000000ULL + q.footprint / (64ULL << 20) * 1000000ULL;
        return;
    }
    const bos_request& r = q.r;
    char* region = base + q.off;
    const size_t scratch = scratch_bytes(r);
    bos::ctx_bind_arena(s.ctx, region + scratch, q.footprint - scratch, stream);
    q.dLdI = (float*)region;
    q.order = admitted++;
    q.ev = s.ev;
    q.ev_hand = s.ev_hand;
    q.ev_build = s.ev_build;
    q.handed = q.built = false;
    void* st = (void*)stream;
    // requests of the batched kinds (the ones bos::ctx_batchable accepts)
    const bool batch = (r.grid.prec == BOS_PREC_FP32_COMP || r.grid.prec == BOS_PREC_BF16_COMP) &&
                       (r.integ.integrator == 0 || r.integ.integrator == 2) && r.light.mode != 2 &&
                       r.integ.ckpt_every <= 64 && (!r.target_dev || r.integ.integrator == 2 || seg != nullptr);
    // the field build: on the build stream for a batched request (its first render launch
    // waits for it), else in line with its own launches
    bos_status_t e = bos_set_grid(s.ctx, &r.grid, r.T_dev, batch ? (void*)stream_build : st);
    if (e == BOS_OK && batch && cudaEventRecord(q.ev_build, stream_build) != cudaSuccess) e = BOS_ERR_CUDA;
    if (e == BOS_OK) e = bos_set_geometry(s.ctx, &r.cam, &r.wall, &r.light, r.pattern_dev, &r.integ);
    if (e == BOS_OK && batch && !bos::ctx_batchable(s.ctx)) e = BOS_ERR_CUDA;   // the two tests agree by construction
    if (e == BOS_OK && batch) {
        // its warp tiles join the batched launches
        q.built = true;
        int ntiles = 0;
        e = bos::ctx_batch_render(s.ctx, r.I_dev, r.disp_dev, r.target_dev ? 1 : 0, stream, &q.J, &ntiles, &q.cost);
        if (e == BOS_OK) {
            q.batched = true;
            q.phase = PH_RENDER;
            q.mode = r.grid.prec == BOS_PREC_BF16_COMP ? 2 : 1;
            q.integ = r.integ.integrator;
            q.tiles[0] = q.tiles[1] = ntiles;
            q.next[0] = q.next[1] = 0;
            return;
        }
    } else if (e == BOS_OK) {
        // its own launches, in admission order on the same stream
        e = bos_render(s.ctx, r.I_dev, r.disp_dev, nullptr, r.target_dev ? 1 : 0, st);
        if (e == BOS_OK && r.target_dev) {
            e = bos_loss_l2(r.I_dev, r.target_dev, (int64_t)r.cam.width * r.cam.height, r.loss_dev, q.dLdI, st);
            if (e == BOS_OK) e = bos_backward(s.ctx, q.dLdI, r.dLdT_dev, st);
        }
        if (e == BOS_OK && cudaEventRecord(q.ev, stream) != cudaSuccess) e = BOS_ERR_CUDA;
        if (e == BOS_OK) {
            q.phase = PH_FINISH;
            return;
        }
    }
    fail_request(q, e);
}

// The request's tiles of its current phase are all enqueued: what follows them.
void bos_server::after_phase(Req& q) {
    Slot& s = *slots[q.slot];
    const bos_request& r = q.r;
    bos_status_t e = BOS_OK;
    if (q.phase == PH_RENDER && r.target_dev) {
        e = bos_loss_l2(r.I_dev, r.target_dev, (int64_t)r.cam.width * r.cam.height, r.loss_dev, q.dLdI, (void*)stream);
        if (e == BOS_OK) e = bos::ctx_batch_backward(s.ctx, q.dLdI, stream, &q.J);
        if (e == BOS_OK && cudaEventRecord(q.ev_hand, stream) != cudaSuccess) e = BOS_ERR_CUDA;
        if (e == BOS_OK) {
            q.phase = PH_ADJOINT;
            q.handed = true;
            return;
        }
    } else if (q.phase == PH_ADJOINT) {
        e = bos::ctx_gradient(s.ctx, r.dLdT_dev, stream_adj);
        if (e == BOS_OK && cudaEventRecord(q.ev, stream_adj) != cudaSuccess) e = BOS_ERR_CUDA;
    } else if (cudaEventRecord(q.ev, stream) != cudaSuccess) {
        e = BOS_ERR_CUDA;
    }
    if (e != BOS_OK) {
        fail_request(q, e);
        return;
    }
    q.phase = PH_FINISH;
}

// Enqueue one batched launch of `phase` (render on stream 0, adjoint on stream 1): the
// kernel variant of the oldest request with tiles of that phase to run, and tiles of the
// requests of that kind, oldest first, up to the launch's work budget (every request in the
// launch gets at least one warp tile).
bool bos_server::launch_batch(int phase) {
    Batch* b = nullptr;
    int inflight = 0;
    for (auto& x : batches) {
        if (x.busy && x.phase == phase) ++inflight;
        else if (!x.busy && !b) b = &x;
    }
    if (!b || inflight >= kInFlight) return false;
    Req* head = nullptr;
    for (uint64_t tk : active) {
        Req& q = reqs[tk];
        if (q.batched && q.phase == phase && q.next[phase] < q.tiles[phase]) {
            head = &q;
            break;
        }
    }
    if (!head) return false;
    const int mode = head->mode, integ = head->integ;
    cudaStream_t st = phase == PH_RENDER ? stream : stream_adj;
    const double budget = phase == PH_RENDER ? kRenderBudget : kAdjointBudget;
    std::vector<Req*> sel;
    std::vector<int> take;
    double used = 0.0;
    for (uint64_t tk : active) {
        if (used >= budget || (int)sel.size() >= kMaxBatchJobs) break;
        Req& q = reqs[tk];
        if (!(q.batched && q.phase == phase && q.mode == mode && q.integ == integ && q.next[phase] < q.tiles[phase]))
            continue;
        const int rem = q.tiles[phase] - q.next[phase];
        const int n = (int)std::min<double>(rem, std::max(1.0, (budget - used) / q.cost));
        sel.push_back(&q);
        take.push_back(n);
        used += n * q.cost;
    }
    int total = 0, k_max = 1;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < sel.size(); ++i) {
        Req& q = *sel[i];
        if (phase == PH_ADJOINT && q.handed) {   // its render phase and L_BOS ran on stream 0
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, q.ev_hand, 0);
            q.handed = false;
        }
        if (phase == PH_RENDER && q.built) {     // its field build ran on the build stream
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, q.ev_build, 0);
            q.built = false;
        }
        bos::BatchJob& J = b->host[i];
        J = q.J;
        J.tile0 = q.next[phase];
        J.first = total;
        total += take[i];
        q.next[phase] += take[i];
        k_max = std::max(k_max, q.J.ck.every);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->dev, b->host, sel.size() * sizeof(bos::BatchJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->counter, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = phase == PH_RENDER ? bos::launch_render_batch(mode, integ, b->dev, (int)sel.size(), total, b->counter,
                                                          num_sms, st)
                               : bos::launch_adjoint_batch(mode, integ, b->dev, (int)sel.size(), total, b->counter, seg,
                                                           integ == 2 ? 1 : kSegK, num_sms, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev, st);
    b->busy = true;
    b->phase = phase;
    ++n_batches;
    n_batch_tiles += (uint64_t)total;
    n_batch_jobs += sel.size();
    max_batch_jobs = std::max(max_batch_jobs, (int)sel.size());
    for (Req* q : sel) {
        if (e != cudaSuccess) fail_request(*q, BOS_ERR_CUDA);
        else if (q->next[phase] == q->tiles[phase]) after_phase(*q);
    }
    return e == cudaSuccess;
}

void bos_server::finish(Slot& s) {
    Req& q = reqs[s.ticket];
    q.t_done = s.t_finished.load();
    if (!fake() && q.status == BOS_OK) {
        bos_status_t st = bos_status(s.ctx);
        if (st != BOS_OK) q.status = st;
    }
    arena.release(q.off, q.footprint);
    q.done = true;
    s.busy = false;
    s.finished.store(false);
    active.erase(std::remove(active.begin(), active.end(), s.ticket), active.end());
}

void bos_server::run() {
    if (!fake()) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool any_busy = false;
        const uint64_t t = now_ns();
        if (!fake())
            for (auto& x : batches)
                if (x.busy && cudaEventQuery(x.ev) == cudaSuccess) x.busy = false;
        for (auto& sp : slots) {
            Slot& s = *sp;
            if (s.busy && fake() && !s.finished.load() && t >= s.fake_due) {
                s.t_finished.store(t);
                s.finished.store(true);
            }
            if (s.busy && !fake() && !s.finished.load()) {
                Req& q = reqs[s.ticket];
                if (q.phase == PH_FINISH && cudaEventQuery(q.ev) == cudaSuccess) {
                    s.t_finished.store(now_ns());
                    s.finished.store(true);
                }
            }
            if (s.busy && s.finished.load()) finish(s);
            any_busy = any_busy || s.busy;
        }
        // admit in arrival order while a slot and the memory are free
        while (!pending.empty()) {
            Slot* free_slot = nullptr;
            for (auto& sp : slots)
                if (!sp->busy) {
                    free_slot = sp.get();
                    break;
                }
            if (!free_slot) break;
            const uint64_t tk = pending.front();
            Req& q = reqs[tk];
            size_t off;
            if (!arena.alloc(q.footprint, &off)) break;
            pending.pop_front();
            q.off = off;
            q.t_admit = now_ns();
            for (size_t i = 0; i < slots.size(); ++i)
                if (slots[i].get() == free_slot) q.slot = (int)i;
            free_slot->busy = true;
            free_slot->ticket = tk;
            any_busy = true;
            if (arena.used() > peak_used) peak_used = arena.used();
            active.push_back(tk);
            launch(q, *free_slot);
        }
        if (!fake())
            for (int ph = PH_RENDER; ph <= PH_ADJOINT; ++ph)
                while (launch_batch(ph)) {
                }
        cv.notify_all();
        if (stop && pending.empty() && !any_busy) break;
        cv.wait_for(lk, std::chrono::microseconds(fake() ? 200 : 100));
    }
}

extern "C" {

bos_status_t bos_request_footprint(const bos_request* r, uint64_t* bytes) {
    if (!bytes || validate_request(r) != BOS_OK) return BOS_ERR_INVALID_ARG;
    *bytes = bos::request_bytes(r->grid, r->cam, r->light, r->integ, r->target_dev != nullptr) + scratch_bytes(*r);
    return BOS_OK;
}

namespace {

// Release every CUDA resource of a server (after its stream has drained).
void release_gpu(bos_server* s) {
    for (auto& o : s->slots) {
        if (o->ctx) {
            bos::ctx_bind_arena(o->ctx, nullptr, 0, s->stream);
            bos_destroy(o->ctx);
        }
        if (o->ev) cudaEventDestroy(o->ev);
        if (o->ev_hand) cudaEventDestroy(o->ev_hand);
        if (o->ev_build) cudaEventDestroy(o->ev_build);
    }
    for (auto& b : s->batches) {
        if (b.ev) cudaEventDestroy(b.ev);
        if (b.host) cudaFreeHost(b.host);
        if (b.dev) cudaFree(b.dev);
        if (b.counter) cudaFree(b.counter);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->stream_adj) cudaStreamDestroy(s->stream_adj);
    if (s->stream_build) cudaStreamDestroy(s->stream_build);
    if (s->base) cudaFree(s->base);
}

}  // namespace

bos_status_t bos_server_create(bos_server** out, int device, uint64_t mem_limit_bytes, int nslots, int flags) {
    if (!out || nslots < 1 || nslots > kMaxBatchJobs || mem_limit_bytes < (1u << 20)) return BOS_ERR_INVALID_ARG;
    *out = nullptr;
    std::unique_ptr<bos_server> s(new bos_server());
    s->device = device;
    s->flags = flags;
    s->limit = mem_limit_bytes;
    s->arena.reset(mem_limit_bytes);
    for (int i = 0; i < nslots; ++i) {
        std::unique_ptr<Slot> sl(new Slot());
        sl->owner = s.get();
        s->slots.push_back(std::move(sl));
    }
    if (!s->fake()) {
        int prev = 0;
        cudaGetDevice(&prev);
        if (cudaSetDevice(device) != cudaSuccess) return BOS_ERR_INVALID_ARG;
        bos_status_t st = BOS_OK;
        if (cudaMalloc((void**)&s->base, mem_limit_bytes) != cudaSuccess) {
            cudaGetLastError();
            s->base = nullptr;
            st = BOS_ERR_OOM;
        }
        if (st == BOS_OK && (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
                             cudaStreamCreateWithFlags(&s->stream_adj, cudaStreamNonBlocking) != cudaSuccess ||
                             cudaStreamCreateWithFlags(&s->stream_build, cudaStreamNonBlocking) != cudaSuccess))
            st = BOS_ERR_CUDA;
        if (st == BOS_OK) cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
        for (auto& b : s->batches) {
            if (st != BOS_OK) break;
            if (cudaHostAlloc((void**)&b.host, kMaxBatchJobs * sizeof(bos::BatchJob), cudaHostAllocDefault) != cudaSuccess ||
                cudaMalloc((void**)&b.dev, kMaxBatchJobs * sizeof(bos::BatchJob)) != cudaSuccess ||
                cudaMalloc((void**)&b.counter, sizeof(int)) != cudaSuccess ||
                cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess)
                st = BOS_ERR_CUDA;
        }
        for (auto& o : s->slots) {
            if (st != BOS_OK) break;
            if (cudaEventCreateWithFlags(&o->ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&o->ev_hand, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&o->ev_build, cudaEventDisableTiming) != cudaSuccess)
                st = BOS_ERR_CUDA;
            if (st == BOS_OK) st = bos_create(&o->ctx, device, 0);
            if (st == BOS_OK) bos::ctx_bind_arena(o->ctx, nullptr, 0, s->stream);
        }
        // segment slices of the batched Sharma adjoint, carved once from the arena when it is
        // large enough (otherwise forward + adjoint requests of that kind run their own launches)
        const size_t seg_bytes = bos::adjoint_segment_bytes(kSegK);
        size_t off = 0;
        if (st == BOS_OK && mem_limit_bytes >= 4 * seg_bytes && s->arena.alloc(seg_bytes, &off)) {
            s->seg = (float*)(s->base + off);
            s->peak_used = s->arena.used();
        }
        if (st == BOS_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = BOS_ERR_CUDA;
        if (st != BOS_OK) {
            cudaGetLastError();
            release_gpu(s.get());
            cudaSetDevice(prev);
            return st;
        }
        cudaSetDevice(prev);
    }
    bos_server* raw = s.release();
    raw->sched = std::thread([raw] { raw->run(); });
    *out = raw;
    return BOS_OK;
}

bos_status_t bos_submit(bos_server* s, const bos_request* r, uint64_t* ticket) {
    if (!s || !ticket) return BOS_ERR_INVALID_ARG;
    bos_status_t v = validate_request(r);
    if (v != BOS_OK) return v;
    uint64_t fp = bos::request_bytes(r->grid, r->cam, r->light, r->integ, r->target_dev != nullptr) + scratch_bytes(*r);
    if (bos::align_up(fp) > s->limit) return BOS_ERR_ADMISSION;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return BOS_ERR_NOT_READY;
    uint64_t t = s->next_ticket++;
    Req& q = s->reqs[t];
    q.r = *r;
    q.footprint = fp;
    q.t_submit = now_ns();
    s->pending.push_back(t);
    *ticket = t;
    s->cv.notify_all();
    return BOS_OK;
}

bos_status_t bos_wait(bos_server* s, uint64_t ticket, uint64_t timeout_ns) {
    if (!s) return BOS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return BOS_ERR_INVALID_ARG;
    const auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns);
    while (!it->second.done) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done) return BOS_ERR_TIMEOUT;
    }
    return (bos_status_t)it->second.status;
}

bos_status_t bos_ticket(bos_server* s, uint64_t ticket, bos_ticket_info* info) {
    if (!s || !info) return BOS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return BOS_ERR_INVALID_ARG;
    const Req& q = it->second;
    info->submit_ns = q.t_submit;
    info->admit_ns = q.t_admit;
    info->done_ns = q.t_done;
    info->footprint_bytes = q.footprint;
    info->status = q.done ? q.status : BOS_ERR_NOT_READY;
    info->done = q.done ? 1 : 0;
    info->slot = q.slot;
    return BOS_OK;
}

bos_status_t bos_server_stats(bos_server* s, uint64_t* arena_bytes, uint64_t* peak_used_bytes, int* queued,
                              int* running) {
    if (!s) return BOS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (arena_bytes) *arena_bytes = s->limit;
    if (peak_used_bytes) *peak_used_bytes = s->peak_used;
    if (queued) *queued = (int)s->pending.size();
    if (running) {
        int n = 0;
        for (auto& sp : s->slots) n += sp->busy ? 1 : 0;
        *running = n;
    }
    return BOS_OK;
}

bos_status_t bos_server_batches(bos_server* s, uint64_t* launches, uint64_t* tiles, uint64_t* job_shares,
                                int* max_jobs) {
    if (!s) return BOS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (launches) *launches = s->n_batches;
    if (tiles) *tiles = s->n_batch_tiles;
    if (job_shares) *job_shares = s->n_batch_jobs;
    if (max_jobs) *max_jobs = s->max_batch_jobs;
    return BOS_OK;
}

bos_status_t bos_server_destroy(bos_server* s, uint64_t timeout_ns) {
    if (!s) return BOS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    // wait (bounded) for the queue to drain and the running requests to finish
    const auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns);
    bool drained = false;
    while (Clock::now() < deadline) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            bool busy = !s->pending.empty();
            for (auto& sp : s->slots) busy = busy || sp->busy;
            if (!busy) {
                drained = true;
                break;
            }
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    if (!drained) return BOS_ERR_TIMEOUT;   // the server stays alive; the caller may retry
    s->sched.join();
    if (!s->fake()) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(s->device);
        cudaStreamSynchronize(s->stream);
        cudaStreamSynchronize(s->stream_adj);
        cudaStreamSynchronize(s->stream_build);
        release_gpu(s);
        cudaSetDevice(prev);
    }
    delete s;
    return BOS_OK;
}

}  // extern "C"
