// Request server: continuous batching of forward and forward+adjoint renders on one GPU.
//
// Requests arrive at any time (bos_submit, from any thread) and queue FIFO.  A scheduler
// thread admits the queue head as soon as (a) one of the server's slots is free and
// (b) the request's exact device footprint fits in the free space of the server's arena,
// a single device allocation of mem_limit_bytes made once at creation (first-fit with
// coalescing; nothing is allocated or freed per request).  An admitted request runs on its
// slot's own non-blocking stream and context (field build, render, loss, backward), so the
// kernels of all admitted requests overlap on the device, and requests that arrive while
// others run are admitted as soon as slots and memory free up.  A host function enqueued
// behind the request's last kernel marks its completion; every wait is bounded.
//
// The fake executor (BOS_SERVER_FAKE_EXECUTOR) runs the same admission, slot and memory
// logic without any CUDA call: an admitted request "runs" for a time proportional to
// its footprint.  It exists to test the scheduler on machines without a GPU.
#include <math.h>
#include <stdio.h>
#include <string.h>

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

struct Req {
    bos_request r;
    uint64_t footprint = 0;
    uint64_t t_submit = 0, t_admit = 0, t_done = 0;
    int status = BOS_OK;
    int slot = -1;
    bool done = false;
    size_t off = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    bos_ctx* ctx = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    std::atomic<bool> finished{false};
    std::atomic<uint64_t> t_finished{0};
    uint64_t fake_due = 0;
    struct bos_server* owner = nullptr;
};

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

    bool fake() const { return flags & BOS_SERVER_FAKE_EXECUTOR; }
    void run();
    void launch(Req& q, Slot& s);
    void finish(Slot& s);
};

namespace {

void CUDART_CB on_done(void* arg) {
    // Runs on a driver thread: no CUDA calls here, only flags and a wake-up.
    Slot* s = static_cast<Slot*>(arg);
    s->t_finished.store(now_ns());
    s->finished.store(true);
    s->owner->cv.notify_all();
}

bos_status_t validate_request(const bos_request* r) {
    if (!r || !r->T_dev || !r->pattern_dev || !r->I_dev) return BOS_ERR_INVALID_ARG;
    if (r->target_dev && (!r->loss_dev || !r->dLdT_dev)) return BOS_ERR_INVALID_ARG;
    // the checks of bos_set_grid / bos_set_geometry, at submission rather than at launch
    bos_status_t e = bos::check_grid_desc(&r->grid, "bos_submit");
    if (e == BOS_OK) e = bos::check_geometry_desc(&r->cam, &r->wall, &r->light, r->pattern_dev, &r->integ, "bos_submit");
    return e;
}

}  // namespace

void bos_server::launch(Req& q, Slot& s) {
    if (fake()) {
        // simulated run time: 1 ms + 1 ms per 64 MiB of footprint
        s.fake_due = now_ns() + 1000000ULL + q.footprint / (64ULL << 20) * 1000000ULL;
        return;
    }
    const bos_request& r = q.r;
    char* region = base + q.off;
    size_t scratch = scratch_bytes(r);
    bos::ctx_bind_arena(s.ctx, region + scratch, q.footprint - scratch, s.stream);
    float* dLdI = (float*)region;
    void* st = (void*)s.stream;
    bos_status_t e = bos_set_grid(s.ctx, &r.grid, r.T_dev, st);
    if (e == BOS_OK) e = bos_set_geometry(s.ctx, &r.cam, &r.wall, &r.light, r.pattern_dev, &r.integ);
    if (e == BOS_OK) e = bos_render(s.ctx, r.I_dev, r.disp_dev, nullptr, r.target_dev ? 1 : 0, st);
    if (e == BOS_OK && r.target_dev) {
        e = bos_loss_l2(r.I_dev, r.target_dev, (int64_t)r.cam.width * r.cam.height, r.loss_dev, dLdI, st);
        if (e == BOS_OK) e = bos_backward(s.ctx, dLdI, r.dLdT_dev, st);
    }
    if (e == BOS_OK && cudaLaunchHostFunc(s.stream, on_done, &s) != cudaSuccess) e = BOS_ERR_CUDA;
    if (e != BOS_OK) {
        q.status = e;
        // let the work already enqueued drain before the memory is reused
        cudaStreamSynchronize(s.stream);
        s.t_finished.store(now_ns());
        s.finished.store(true);
    }
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
}

void bos_server::run() {
    if (!fake()) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool any_busy = false;
        const uint64_t t = now_ns();
        for (auto& sp : slots) {
            Slot& s = *sp;
            if (s.busy && fake() && !s.finished.load() && t >= s.fake_due) {
                s.t_finished.store(t);
                s.finished.store(true);
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
            launch(q, *free_slot);
        }
        cv.notify_all();
        if (stop && pending.empty() && !any_busy) break;
        cv.wait_for(lk, std::chrono::microseconds(fake() ? 200 : 500));
    }
}

extern "C" {

bos_status_t bos_request_footprint(const bos_request* r, uint64_t* bytes) {
    if (!bytes || validate_request(r) != BOS_OK) return BOS_ERR_INVALID_ARG;
    *bytes = bos::request_bytes(r->grid, r->cam, r->light, r->integ, r->target_dev != nullptr) + scratch_bytes(*r);
    return BOS_OK;
}

bos_status_t bos_server_create(bos_server** out, int device, uint64_t mem_limit_bytes, int nslots, int flags) {
    if (!out || nslots < 1 || nslots > 64 || mem_limit_bytes < (1u << 20)) return BOS_ERR_INVALID_ARG;
    *out = nullptr;
    std::unique_ptr<bos_server> s(new bos_server());
    s->device = device;
    s->flags = flags;
    s->limit = mem_limit_bytes;
    s->arena.reset(mem_limit_bytes);
    if (!s->fake()) {
        int prev = 0;
        cudaGetDevice(&prev);
        if (cudaSetDevice(device) != cudaSuccess) return BOS_ERR_INVALID_ARG;
        if (cudaMalloc((void**)&s->base, mem_limit_bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaSetDevice(prev);
            return BOS_ERR_OOM;
        }
        cudaSetDevice(prev);
    }
    for (int i = 0; i < nslots; ++i) {
        std::unique_ptr<Slot> sl(new Slot());
        sl->owner = s.get();
        if (!s->fake()) {
            int prev = 0;
            cudaGetDevice(&prev);
            cudaSetDevice(device);
            cudaError_t e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
            cudaSetDevice(prev);
            bos_status_t st = e == cudaSuccess ? bos_create(&sl->ctx, device, 0) : BOS_ERR_CUDA;
            if (st != BOS_OK) {
                for (auto& o : s->slots) {
                    if (o->ctx) bos_destroy(o->ctx);
                    if (o->stream) cudaStreamDestroy(o->stream);
                }
                if (sl->stream) cudaStreamDestroy(sl->stream);
                cudaFree(s->base);
                return st;
            }
            bos::ctx_bind_arena(sl->ctx, nullptr, 0, sl->stream);
        }
        s->slots.push_back(std::move(sl));
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
        for (auto& sp : s->slots) {
            if (sp->stream) cudaStreamSynchronize(sp->stream);
            if (sp->ctx) {
                bos::ctx_bind_arena(sp->ctx, nullptr, 0, sp->stream);
                bos_destroy(sp->ctx);
            }
            if (sp->stream) cudaStreamDestroy(sp->stream);
        }
        if (s->base) cudaFree(s->base);
    }
    delete s;
    return BOS_OK;
}

}  // extern "C"
