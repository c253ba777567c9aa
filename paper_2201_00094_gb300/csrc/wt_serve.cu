// Serving runtime: continuous batching of Wavelet OIT frames on one GPU.
//
// Frames (requests) are submitted from any host thread.  A scheduler thread
// admits them in arrival order while a slot is free and the accounted bytes
// (fragments + coefficients + output) stay under the memory cap, keeps each
// admitted frame's coefficient buffer resident in a device arena, and runs
// steps: one persistent kernel per step over a task table that gives every
// admitted, unfinished frame an equal share of the step's tile budget.
// Frames that arrive while others are on the GPU join the next step, so their
// tiles run in the same launches as the older frames' remaining tiles.
// Completion is marked by a CUDA event after the step that ran a frame's last
// tile.  Every host wait is bounded; kernels never wait on the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wt.h"
#include "wt_internal.h"
#include "wt_planner.h"
#include "wt_trace.h"
#include "wt_tile.cuh"

namespace wt {

// The planner (admission and step planning) is host-only: wt_planner.h.

// ---------------------------------------------------------------- device arena

// First-fit allocator over one device allocation made at server creation.
class Arena {
  public:
    bool init(size_t bytes) {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) return false;
        free_[0] = bytes;
        size_ = bytes;
        return true;
    }
    void destroy() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    void *alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_[off] = bytes;
                return static_cast<char *>(base_) + off;
            }
        }
        return nullptr;
    }
    void free(void *p) {
        if (!p) return;
        const size_t off = static_cast<char *>(p) - static_cast<char *>(base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t len = u->second, start = off;
        used_.erase(u);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }

  private:
    void *base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_, used_;
};

// ---------------------------------------------------------------- server

namespace {
double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}
int64_t ntiles(const wt_desc *d) {
    return (int64_t)((d->width + d->tile_w - 1) / d->tile_w) * ((d->height + d->tile_h - 1) / d->tile_h);
}
}  // namespace

struct ServerImpl {
    wt_serve_config cfg;
    int device = 0, sms = 1, occupancy = 1;
    cudaStream_t stream = nullptr;
    Planner *planner = nullptr;
    Arena arena;
    Params *d_slots = nullptr, *h_slots = nullptr;  // h_slots pinned
    static constexpr int kRing = 2;                  // task tables in flight
    ServeTask *d_tasks[kRing] = {}, *h_tasks[kRing] = {};
    cudaEvent_t ring_free[kRing] = {};
    unsigned long long *d_counter[kRing] = {};
    int max_tasks = 0;
    int ring = 0;
    cudaEvent_t t0_event = nullptr;
    double t0_host = 0;
    unsigned long long *err = nullptr;

    struct Req {
        wt_desc desc;
        Params params;
        void *coeff = nullptr;
        size_t coeff_bytes = 0;
        cudaEvent_t done_ev = nullptr;
        cudaEvent_t ready_ev = nullptr;  // inputs and output ready on the producer's stream
        bool scheduled = false, done = false;
        double t_submit = 0, t_admit = 0, t_done = 0;
    };
    std::unordered_map<int64_t, Req> reqs;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    wt_status fault = WT_OK;

    void run();
    bool step_locked(std::unique_lock<std::mutex> &lk);
    void poll_locked();
};

extern unsigned long long *error_word();  // wt_api.cu

void ServerImpl::poll_locked() {
    for (auto &kv : reqs) {
        Req &r = kv.second;
        if (r.scheduled && !r.done && cudaEventQuery(r.done_ev) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0_event, r.done_ev);
            r.t_done = t0_host + 1000.0 * ms;
            r.done = true;
            cv.notify_all();
        }
    }
}

bool ServerImpl::step_locked(std::unique_lock<std::mutex> &lk) {
    std::vector<int64_t> admitted;
    // coefficient buffers come from the arena; a refusal (fragmentation only:
    // the arena is as large as the cap) leaves the request at the queue head
    planner->admit(admitted, [&](int64_t id) {
        Req &r = reqs[id];
        r.coeff = arena.alloc(r.coeff_bytes);
        return r.coeff != nullptr;
    });
    for (int64_t id : admitted) {
        Req &r = reqs[id];
        r.t_admit = now_us();
        r.params.coeff = r.coeff;
        // the request's work runs after what its producer enqueued before submitting
        if (cudaStreamWaitEvent(stream, r.ready_ev, 0) != cudaSuccess) {
            fault = WT_ERR_CUDA;
            return false;
        }
        const int slot = planner->slot_of(id);
        h_slots[slot] = r.params;
        if (cudaMemcpyAsync(d_slots + slot, h_slots + slot, sizeof(Params), cudaMemcpyHostToDevice,
                            stream) != cudaSuccess) {
            fault = WT_ERR_CUDA;
            return false;
        }
    }
    std::vector<Planner::Range> ranges;
    std::vector<int64_t> finishing;
    planner->plan(ranges, finishing);
    if (ranges.empty() && finishing.empty()) return false;
    if (!ranges.empty()) {
        const int b = ring;
        ring = (ring + 1) % kRing;
        // the host table of this ring entry is reused only after its copy ran
        cudaEventSynchronize(ring_free[b]);
        int64_t total = 0;
        if ((int)ranges.size() > max_tasks) {  // one range per slot by construction
            fault = WT_ERR_ARG;
            return false;
        }
        const int nt = (int)ranges.size();
        for (int i = 0; i < nt; ++i) {
            h_tasks[b][i].slot = ranges[i].slot;
            h_tasks[b][i].tile0 = ranges[i].tile0;
            h_tasks[b][i].start = total;
            total += ranges[i].count;
        }
        cudaError_t e = cudaMemcpyAsync(d_tasks[b], h_tasks[b], nt * sizeof(ServeTask),
                                        cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaEventRecord(ring_free[b], stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_counter[b], 0, sizeof(unsigned long long), stream);
        const int npx = cfg.tile_w * cfg.tile_h;
        const int grid = (int)std::min<int64_t>(total, (int64_t)sms * occupancy);
        const ServeLaunch *L = by_dtype(cfg.coeff_dtype, kServe0, kServe1, kServe2, kServe3);
        if (e == cudaSuccess) e = L[cfg.J - 1](d_slots, d_tasks[b], nt, total, d_counter[b], npx, grid, stream);
        if (e != cudaSuccess) {
            fault = WT_ERR_CUDA;
            return false;
        }
    }
    for (int64_t id : finishing) {
        Req &r = reqs[id];
        cudaEventRecord(r.done_ev, stream);
        r.scheduled = true;
    }
    (void)lk;
    return true;
}

void ServerImpl::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        poll_locked();
        const bool launched = fault == WT_OK && step_locked(lk);
        poll_locked();
        if (!launched) {
            // nothing to launch: wait (bounded) for a submission, a release or
            // the completion of in-flight work
            cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace wt

using namespace wt;

struct wt_server {
    ServerImpl impl;
};
struct wt_planner {
    Planner *p;
};

extern "C" {

wt_status wt_serve_create(const wt_serve_config *cfg, wt_server **out) {
    WT_TRACE();
    if (!cfg || !out) return WT_ERR_ARG;
    if (cfg->J < 1 || cfg->J > kMaxJ || (cfg->coeff_dtype != WT_F32 && cfg->coeff_dtype != WT_BF16 &&
                                     cfg->coeff_dtype != WT_F16 && cfg->coeff_dtype != WT_SE16))
        return WT_ERR_UNSUPPORTED;
    if (cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->mem_cap_bytes <= 0 || cfg->step_tiles < 1 ||
        cfg->tile_w < 1 || cfg->tile_h < 1 || (int64_t)cfg->tile_w * cfg->tile_h > kMaxTilePx)
        return WT_ERR_ARG;
    wt_server *s = new wt_server();
    ServerImpl &S = s->impl;
    S.cfg = *cfg;
    if (cudaGetDevice(&S.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&S.sms, cudaDevAttrMultiProcessorCount, S.device) != cudaSuccess) {
        delete s;
        return WT_ERR_CUDA;
    }
    const ServeOccupancy *O = by_dtype(cfg->coeff_dtype, kServeOcc0, kServeOcc1, kServeOcc2, kServeOcc3);
    S.occupancy = std::max(1, O[cfg->J - 1](cfg->tile_w * cfg->tile_h));
    S.max_tasks = cfg->max_slots;
    S.err = error_word();
    bool ok = S.err != nullptr;
    ok = ok && cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && S.arena.init((size_t)cfg->mem_cap_bytes);
    ok = ok && cudaMalloc(&S.d_slots, sizeof(Params) * cfg->max_slots) == cudaSuccess;
    ok = ok && cudaMallocHost(&S.h_slots, sizeof(Params) * cfg->max_slots) == cudaSuccess;
    for (int b = 0; b < ServerImpl::kRing && ok; ++b) {
        ok = ok && cudaMalloc(&S.d_tasks[b], sizeof(ServeTask) * S.max_tasks) == cudaSuccess;
        ok = ok && cudaMallocHost(&S.h_tasks[b], sizeof(ServeTask) * S.max_tasks) == cudaSuccess;
        ok = ok && cudaMalloc(&S.d_counter[b], sizeof(unsigned long long)) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&S.ring_free[b], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventRecord(S.ring_free[b], S.stream) == cudaSuccess;
    }
    ok = ok && cudaEventCreate(&S.t0_event) == cudaSuccess;
    ok = ok && cudaEventRecord(S.t0_event, S.stream) == cudaSuccess;
    ok = ok && cudaEventSynchronize(S.t0_event) == cudaSuccess;
    if (!ok) {
        wt_serve_destroy(s);
        return WT_ERR_CUDA;
    }
    S.t0_host = now_us();
    S.planner = new Planner(cfg->max_slots, cfg->mem_cap_bytes, cfg->step_tiles);
    S.worker = std::thread([&S] { S.run(); });
    *out = s;
    return WT_OK;
}

wt_status wt_serve_submit(wt_server *s, const wt_desc *d, const wt_frags *f, const float bg[3],
                          float *out, wt_stream ready_stream, int64_t *request_id) {
    WT_TRACE();
    if (!s || !d || !f || !bg || !out || !request_id) return WT_ERR_ARG;
    ServerImpl &S = s->impl;
    if (d->J != S.cfg.J || d->coeff_dtype != S.cfg.coeff_dtype || d->flags != S.cfg.flags ||
        d->tile_w != S.cfg.tile_w || d->tile_h != S.cfg.tile_h)
        return WT_ERR_UNSUPPORTED;
    if (d->width < 1 || d->height < 1 || (int64_t)d->width * d->height >= (int64_t(1) << 31) ||
        d->reserved != 0)
        return WT_ERR_ARG;
    if (f->n < 0 || !f->tile_offsets || (f->n > 0 && (!f->pixel || !f->z || !f->alpha || !f->r ||
                                                       !f->g || !f->b)))
        return WT_ERR_ARG;
    const void *ptrs[7] = {f->pixel, f->z, f->alpha, f->r, f->g, f->b, out};
    for (const void *p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) & 15) return WT_ERR_ARG;
    const int64_t P = (int64_t)d->width * d->height;
    ServerImpl::Req r;
    r.desc = *d;
    r.coeff_bytes = coeff_storage_bytes(P, d->J, d->coeff_dtype);
    Params &p = r.params;
    std::memset(&p, 0, sizeof(p));
    p.g.width = d->width;
    p.g.height = d->height;
    p.g.tile_w = d->tile_w;
    p.g.tile_h = d->tile_h;
    p.g.ntx = (d->width + d->tile_w - 1) / d->tile_w;
    p.flags = d->flags;
    set_row_division(p);
    p.n = f->n;
    p.pixel = f->pixel;
    p.z = f->z;
    p.alpha = f->alpha;
    p.r = f->r;
    p.gc = f->g;
    p.b = f->b;
    p.off = f->tile_offsets;
    p.out = out;
    p.bg0 = bg[0];
    p.bg1 = bg[1];
    p.bg2 = bg[2];
    p.err = S.err;
    const int64_t bytes = f->n * 24 + (ntiles(d) + 1) * 8 + (int64_t)r.coeff_bytes + P * 16;
    if (cudaEventCreate(&r.done_ev) != cudaSuccess) return WT_ERR_CUDA;
    if (cudaEventCreateWithFlags(&r.ready_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r.ready_ev, reinterpret_cast<cudaStream_t>(ready_stream)) != cudaSuccess) {
        cudaEventDestroy(r.done_ev);
        if (r.ready_ev) cudaEventDestroy(r.ready_ev);
        return WT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(S.mu);
    if (S.fault != WT_OK) {
        cudaEventDestroy(r.done_ev);
        cudaEventDestroy(r.ready_ev);
        return S.fault;
    }
    const int64_t id = S.planner->submit(bytes, ntiles(d));
    if (id < 0) {
        cudaEventDestroy(r.done_ev);
        cudaEventDestroy(r.ready_ev);
        return (wt_status)(-id);
    }
    r.t_submit = now_us();
    S.reqs[id] = r;
    *request_id = id;
    S.cv.notify_all();
    return WT_OK;
}

wt_status wt_serve_wait(wt_server *s, int64_t id, int64_t timeout_us) {
    WT_TRACE();
    if (!s || timeout_us < 0) return WT_ERR_ARG;
    ServerImpl &S = s->impl;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) return WT_ERR_ARG;
    const bool ok = S.cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
        auto jt = S.reqs.find(id);
        return jt == S.reqs.end() || jt->second.done || S.fault != WT_OK;
    });
    if (S.fault != WT_OK) return S.fault;
    return ok ? WT_OK : WT_ERR_TIMEOUT;
}

wt_status wt_serve_query(wt_server *s, int64_t id, wt_serve_info *info) {
    WT_TRACE();
    if (!s || !info) return WT_ERR_ARG;
    ServerImpl &S = s->impl;
    std::lock_guard<std::mutex> g(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) return WT_ERR_ARG;
    const ServerImpl::Req &r = it->second;
    info->state = r.done ? 2 : (r.coeff ? 1 : 0);
    info->submit_us = r.t_submit - S.t0_host;
    info->admit_us = r.coeff ? r.t_admit - S.t0_host : -1.0;
    info->done_us = r.done ? r.t_done - S.t0_host : -1.0;
    info->coeff = r.coeff;
    return WT_OK;
}

wt_status wt_serve_release(wt_server *s, int64_t id) {
    WT_TRACE();
    if (!s) return WT_ERR_ARG;
    ServerImpl &S = s->impl;
    std::lock_guard<std::mutex> g(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end() || !it->second.done) return WT_ERR_ARG;
    S.planner->release(id);
    S.arena.free(it->second.coeff);
    cudaEventDestroy(it->second.done_ev);
    cudaEventDestroy(it->second.ready_ev);
    S.reqs.erase(it);
    S.cv.notify_all();
    return WT_OK;
}

wt_status wt_serve_stats(wt_server *s, int64_t *used_bytes, int64_t *queued, int64_t *active) {
    WT_TRACE();
    if (!s) return WT_ERR_ARG;
    ServerImpl &S = s->impl;
    std::lock_guard<std::mutex> g(S.mu);
    if (!S.planner) return WT_ERR_ARG;
    if (used_bytes) *used_bytes = S.planner->used();
    if (queued) *queued = S.planner->queued();
    if (active) *active = S.planner->active();
    return S.fault;
}

wt_status wt_serve_destroy(wt_server *s) {
    WT_TRACE();
    if (!s) return WT_ERR_ARG;
    ServerImpl &S = s->impl;
    {
        std::lock_guard<std::mutex> g(S.mu);
        S.stop = true;
        S.cv.notify_all();
    }
    if (S.worker.joinable()) S.worker.join();
    if (S.stream) cudaStreamSynchronize(S.stream);
    for (auto &kv : S.reqs) {
        if (kv.second.done_ev) cudaEventDestroy(kv.second.done_ev);
        if (kv.second.ready_ev) cudaEventDestroy(kv.second.ready_ev);
    }
    for (int b = 0; b < ServerImpl::kRing; ++b) {
        if (S.d_tasks[b]) cudaFree(S.d_tasks[b]);
        if (S.h_tasks[b]) cudaFreeHost(S.h_tasks[b]);
        if (S.d_counter[b]) cudaFree(S.d_counter[b]);
        if (S.ring_free[b]) cudaEventDestroy(S.ring_free[b]);
    }
    if (S.d_slots) cudaFree(S.d_slots);
    if (S.h_slots) cudaFreeHost(S.h_slots);
    if (S.t0_event) cudaEventDestroy(S.t0_event);
    S.arena.destroy();
    if (S.stream) cudaStreamDestroy(S.stream);
    delete S.planner;
    delete s;
    return WT_OK;
}

// ---- host-only planner (no GPU needed)

wt_planner *wt_planner_create(int32_t max_slots, int64_t cap, int64_t step_tiles) {
    if (max_slots < 1 || cap <= 0 || step_tiles < 1) return nullptr;
    return new wt_planner{new Planner(max_slots, cap, step_tiles)};
}

int64_t wt_planner_submit(wt_planner *pl, int64_t bytes, int64_t tiles) {
    return pl ? pl->p->submit(bytes, tiles) : -(int64_t)WT_ERR_ARG;
}

int32_t wt_planner_admit(wt_planner *pl, int64_t *ids, int32_t max) {
    if (!pl) return -(int32_t)WT_ERR_ARG;
    std::vector<int64_t> a;
    pl->p->admit(a, [](int64_t) { return true; });
    const int n = std::min<int>((int)a.size(), max);
    for (int i = 0; i < n; ++i) ids[i] = a[i];
    return (int32_t)a.size();
}

int32_t wt_planner_plan(wt_planner *pl, int64_t *ids, int32_t *tile0, int32_t *count, int32_t max,
                        int64_t *finishing, int32_t *nfinishing) {
    if (!pl || !nfinishing) return -(int32_t)WT_ERR_ARG;
    std::vector<Planner::Range> r;
    std::vector<int64_t> fin;
    pl->p->plan(r, fin);
    const int n = std::min<int>((int)r.size(), max);
    for (int i = 0; i < n; ++i) {
        ids[i] = r[i].id;
        tile0[i] = r[i].tile0;
        count[i] = r[i].count;
    }
    const int nf = std::min<int>((int)fin.size(), *nfinishing);
    for (int i = 0; i < nf; ++i) finishing[i] = fin[i];
    *nfinishing = (int32_t)fin.size();
    return (int32_t)r.size();
}

int32_t wt_planner_release(wt_planner *pl, int64_t id) {
    return pl ? (int32_t)pl->p->release(id) : (int32_t)WT_ERR_ARG;
}

int64_t wt_planner_used(const wt_planner *pl) { return pl ? pl->p->used() : -1; }

void wt_planner_destroy(wt_planner *pl) {
    if (!pl) return;
    delete pl->p;
    delete pl;
}

}  // extern "C"
