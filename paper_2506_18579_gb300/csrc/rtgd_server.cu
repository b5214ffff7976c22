// rtgd_server.cu -- request server with continuous batching (host code).
//
// Requests (a grid + a fan + the caller's host output buffer) enter a FIFO.
// The dispatcher thread admits the head request when a stream slot is free
// and the device keeps mem_reserve_bytes free after the request's own needs;
// it queues the trace and the device-to-pinned copy of the records on the
// slot's stream and records an event.  The completion thread polls the
// in-flight events, copies finished records to the caller's buffer and wakes
// the waiters.  Requests therefore join the GPU while others are running.
// With fusion on, mixed-precision requests that would run at four lanes per
// ray on their own are small: the dispatcher admits a small head request
// together with the queued small requests that can share its launch (same
// grid, same integrator) up to fuse_max_rays rays in total, and traces them
// as one four-lane launch (a fused batch occupies one slot).  A GPU that one
// small fan leaves mostly idle is filled by several.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rtgd.h"
#include "rtgd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const rt_grid *grid = nullptr;
    rt_fan_desc fan;
    std::vector<double> freq, el, az;  // copies of the fan arrays
    rt_ray_result *out_host = nullptr;
    size_t n = 0;
    Clock::time_point t_submit, t_admit, t_done;
    rt_err status = RT_OK;
    std::string msg;                   // rt_last_error text of a failed request
    int batch_size = 1;                // requests in the launch that traced this one
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    rt_ray_result *dev = nullptr;   // device records (cudaMallocAsync per admission)
    rt_ray_result *pinned = nullptr;
    size_t pinned_cap = 0;
    std::vector<std::shared_ptr<Request>> reqs;  // the admitted batch (records back to back); empty when free
    bool armed = false;             // the batch's work and event are queued: the completer may poll
};

// At most this many requests share one fused launch.
constexpr int kMaxFused = 256;

}  // namespace

struct rt_server {
    rt_server_config cfg;
    int device = 0;
    std::vector<Slot> slots;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> tickets;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_done;
    std::thread dispatcher, completer;
    uint64_t next_ticket = 1;
    size_t small_limit = 0;  // fusion: largest small request (rays)
    int inflight = 0;
    bool stopping = false;
};

namespace {

double seconds(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

size_t batch_rays(const std::vector<std::shared_ptr<Request>> &b) {
    size_t n = 0;
    for (const auto &r : b) n += r->n;
    return n;
}

void finish_locked(rt_server *s, Slot &slot, rt_err status) {
    const std::string msg = status != RT_OK ? rt_last_error() : "";  // thread-local: keep it for the waiters
    const auto now = Clock::now();
    for (auto &rp : slot.reqs) {
        rp->status = status;
        rp->msg = msg;
        rp->t_done = now;
        rp->done = true;
    }
    slot.reqs.clear();
    slot.armed = false;
    --s->inflight;
    s->cv_done.notify_all();
    s->cv_dispatch.notify_all();
}

// Device memory a batch of n rays from k requests takes while it runs: its
// records (n x 64 bytes, stream-ordered) and the fan tables and launch
// metadata, counted generously (twice the records plus 4 KiB per request).
// The grids it reads are resident and already counted as used memory.
size_t admission_bytes(size_t n, size_t k) { return n * sizeof(rt_ray_result) * 2 + 4096 * k; }

// Free device memory as admission sees it: the caller's budget function if
// one is configured, otherwise cudaMemGetInfo.
size_t free_device_bytes(rt_server *s) {
    if (s->cfg.free_bytes) return s->cfg.free_bytes(s->cfg.free_bytes_user);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    return free_b;
}

// Small requests of a fusing server (always traced by the fused kernel).
bool is_small(const rt_server *s, const Request &r) {
    return s->cfg.fuse_max_rays > 0 && r.fan.precision == RT_MIXED && r.n <= s->small_limit;
}

// Starts the batch of slot sl (called by the dispatcher with the lock released).
rt_err start(rt_server *s, Slot &sl) {
    cudaSetDevice(s->device);
    const size_t n = batch_rays(sl.reqs);
    for (auto &rp : sl.reqs) {
        rp->fan.freq_mhz = rp->freq.data();
        rp->fan.el_deg = rp->el.data();
        rp->fan.az_deg = rp->az.data();
    }
    if (sl.pinned_cap < n) {
        // grow by powers of two: freeing pinned memory synchronises the device
        size_t cap = 1024;
        while (cap < n) cap *= 2;
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned = nullptr;
        sl.pinned_cap = 0;
        if (cudaMallocHost((void **)&sl.pinned, cap * sizeof(rt_ray_result)) != cudaSuccess)
            return rtgd_set_error(RT_ENOMEM, "server: pinned staging allocation failed");
        sl.pinned_cap = cap;
    }
    if (cudaMallocAsync((void **)&sl.dev, n * sizeof(rt_ray_result), sl.stream) != cudaSuccess)
        return rtgd_set_error(RT_ENOMEM, "server: device allocation failed");
    const rt_launch_config &lc = s->cfg.launch;
    rt_err e;
    // a small request runs the fused kernel, alone or not, so its records do
    // not depend on what shares its launch
    if (!is_small(s, *sl.reqs[0])) {
        e = rtgd_queue_trace(sl.reqs[0]->grid, &sl.reqs[0]->fan, sl.dev, n, &lc, sl.stream);
    } else {
        std::vector<const rt_fan_desc *> fans;
        for (const auto &rp : sl.reqs) fans.push_back(&rp->fan);
        e = rtgd_queue_trace_fans(sl.reqs[0]->grid, fans.data(), (int)fans.size(), sl.dev, n, &lc, sl.stream);
    }
    if (e == RT_OK && cudaMemcpyAsync(sl.pinned, sl.dev, n * sizeof(rt_ray_result), cudaMemcpyDeviceToHost,
                                      sl.stream) != cudaSuccess)
        e = rtgd_set_error(RT_ECUDA, "server: result copy failed");
    cudaFreeAsync(sl.dev, sl.stream);
    sl.dev = nullptr;
    if (e == RT_OK && cudaEventRecord(sl.event, sl.stream) != cudaSuccess)
        e = rtgd_set_error(RT_ECUDA, "server: event record failed");
    return e;
}

void dispatch_loop(rt_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_dispatch.wait(lk, [&] {
            return (s->stopping && s->queue.empty()) || (!s->queue.empty() && s->inflight < (int)s->slots.size());
        });
        if (s->queue.empty()) return;  // stopping, nothing left to admit
        // the batch: the head request, and with fusion the queued requests
        // that can share its launch, in queue order, up to fuse_max_rays rays
        std::vector<size_t> pick{0};
        const Request &head = *s->queue.front();
        size_t n_batch = head.n;
        if (is_small(s, head)) {
            for (size_t i = 1; i < s->queue.size() && pick.size() < (size_t)kMaxFused; ++i) {
                const Request &q = *s->queue[i];
                if (!is_small(s, q) || q.grid != head.grid || q.fan.integrator != head.fan.integrator) continue;
                if (n_batch + q.n > (size_t)s->cfg.fuse_max_rays) continue;
                pick.push_back(i);
                n_batch += q.n;
            }
        }
        // admission by device memory: the batch's device scratch must fit
        // above the reserve while other requests run; an idle server admits
        // any batch that fits at all, and refuses (RT_ENOMEM) one that does not
        const size_t need = admission_bytes(n_batch, pick.size());
        lk.unlock();
        const size_t free_b = free_device_bytes(s);
        lk.lock();
        if (free_b < need + s->cfg.mem_reserve_bytes && s->inflight > 0) {
            // wait for a running request to release memory
            s->cv_dispatch.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        if (free_b < need && pick.size() > 1 && admission_bytes(head.n, 1) <= free_b) {
            pick.resize(1);  // nothing runs: the head request goes alone
        } else if (free_b < need) {
            // nothing runs and the head request alone does not fit: refuse it
            // (its fused companions stay queued) without touching the GPU
            auto rp = s->queue.front();
            s->queue.pop_front();
            rp->t_admit = Clock::now();
            rp->batch_size = 1;
            rp->status = RT_ENOMEM;
            char msg[160];
            std::snprintf(msg, sizeof(msg), "server: request needs %zu bytes of device memory, %zu free", need, free_b);
            rp->msg = msg;
            rp->t_done = rp->t_admit;
            rp->done = true;
            s->cv_done.notify_all();
            continue;
        }
        // the queue only grows at its back while the lock was released, so
        // the picked positions are still valid
        std::vector<std::shared_ptr<Request>> batch;
        for (size_t k = pick.size(); k-- > 0;) {
            batch.push_back(s->queue[pick[k]]);
            s->queue.erase(s->queue.begin() + (std::ptrdiff_t)pick[k]);
        }
        std::reverse(batch.begin(), batch.end());
        int idx = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (s->slots[i].reqs.empty()) {
                idx = (int)i;
                break;
            }
        Slot &sl = s->slots[idx];
        sl.reqs = std::move(batch);
        ++s->inflight;
        const auto now = Clock::now();
        for (auto &rp : sl.reqs) {
            rp->t_admit = now;
            rp->batch_size = (int)sl.reqs.size();
        }
        lk.unlock();
        const rt_err e = start(s, sl);
        lk.lock();
        // until start() has recorded the slot's event, a query of that event
        // reports the previous request (or success, if never recorded)
        if (e != RT_OK) finish_locked(s, sl, e);
        else sl.armed = true;
    }
}

void complete_loop(rt_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->stopping && s->inflight == 0 && s->queue.empty()) return;
        bool any = false;
        for (auto &sl : s->slots) {
            if (sl.reqs.empty()) continue;
            any = true;
            if (!sl.armed) continue;  // still being started by the dispatcher
            const cudaError_t q = cudaEventQuery(sl.event);
            if (q == cudaErrorNotReady) continue;
            rt_err st = RT_OK;
            if (q == cudaSuccess) {
                size_t off = 0;
                for (auto &rp : sl.reqs) {
                    std::memcpy(rp->out_host, sl.pinned + off, rp->n * sizeof(rt_ray_result));
                    off += rp->n;
                }
            } else {
                st = rtgd_set_error(RT_ECUDA, cudaGetErrorString(q));
            }
            finish_locked(s, sl, st);
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(any ? 50 : 500));
        lk.lock();
    }
}

}  // namespace

extern "C" {

rt_err rt_server_create(const rt_server_config *cfg, rt_server **out) {
    if (!out) return rtgd_set_error(RT_EINVAL, "out is NULL");
    *out = nullptr;
    rt_server_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (c.max_inflight == 0) c.max_inflight = 8;
    if (c.max_inflight < 1 || c.max_inflight > 64) return rtgd_set_error(RT_EINVAL, "max_inflight must be in 1..64");
    if (c.fuse_max_rays < 0) return rtgd_set_error(RT_EINVAL, "fuse_max_rays must be >= 0");
    if (c.fuse_max_rays > 0 && (c.launch.kernel == RT_KERNEL_PERSISTENT ||
                                (c.launch.lanes_per_ray != 0 && c.launch.lanes_per_ray != 4)))
        return rtgd_set_error(RT_EINVAL, "fusion runs a plain kernel at four lanes per ray");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return rtgd_set_error(RT_EUNSUPPORTED, "no CUDA device available");
    int device = 0;
    cudaGetDevice(&device);
    size_t four_lane = 0;
    if (c.fuse_max_rays > 0) {
        const rt_err e = rtgd_four_lane_limit(device, &c.launch, &four_lane);
        if (e != RT_OK) return e;
    }
    auto *s = new rt_server();
    s->cfg = c;
    s->device = device;
    s->small_limit = std::min(four_lane, (size_t)std::max(c.fuse_max_rays, 0));
    s->slots.resize(c.max_inflight);
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming) != cudaSuccess) {
            for (auto &t : s->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.event) cudaEventDestroy(t.event);
            }
            delete s;
            return rtgd_set_error(RT_ECUDA, "server: stream creation failed");
        }
    }
    s->dispatcher = std::thread(dispatch_loop, s);
    s->completer = std::thread(complete_loop, s);
    *out = s;
    return RT_OK;
}

rt_err rt_server_submit(rt_server *s, const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_host,
                        size_t out_len, uint64_t *ticket) {
    if (!s || !grid || !fan || !out_host || !ticket) return rtgd_set_error(RT_EINVAL, "NULL argument");
    const size_t n = rt_fan_size(fan);
    if (n == 0) return rtgd_set_error(RT_EINVAL, "empty or invalid fan");
    if (out_len < n) return rtgd_set_error(RT_EINVAL, "out_len smaller than the fan");
    if (!fan->freq_mhz || !fan->el_deg || !fan->az_deg) return rtgd_set_error(RT_EINVAL, "fan arrays must not be NULL");
    auto r = std::make_shared<Request>();
    r->grid = grid;
    r->fan = *fan;
    r->freq.assign(fan->freq_mhz, fan->freq_mhz + fan->n_freq);
    r->el.assign(fan->el_deg, fan->el_deg + fan->n_el);
    r->az.assign(fan->az_deg, fan->az_deg + fan->n_az);
    r->out_host = out_host;
    r->n = n;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return rtgd_set_error(RT_EINVAL, "server is stopping");
    r->ticket = s->next_ticket++;
    s->tickets[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv_dispatch.notify_all();
    return RT_OK;
}

rt_err rt_server_wait(rt_server *s, uint64_t ticket, double timeout_s, rt_request_stats *stats) {
    if (!s) return rtgd_set_error(RT_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return rtgd_set_error(RT_EINVAL, "unknown ticket");
    auto r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
            return rtgd_set_error(RT_ETIMEOUT, "request not finished in time");
    } else {
        s->cv_done.wait(lk, pred);
    }
    s->tickets.erase(it);
    if (stats) {
        stats->queue_s = seconds(r->t_submit, r->t_admit);
        stats->run_s = seconds(r->t_admit, r->t_done);
        stats->total_s = seconds(r->t_submit, r->t_done);
        stats->n_rays = (int64_t)r->n;
        stats->status = r->status;
        stats->batch_size = r->batch_size;
    }
    if (r->status != RT_OK) return rtgd_set_error(r->status, r->msg.c_str());
    return r->status;
}

rt_err rt_server_destroy(rt_server *s) {
    if (!s) return RT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv_dispatch.notify_all();
    }
    s->dispatcher.join();
    s->completer.join();
    for (auto &sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.event);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    delete s;
    return RT_OK;
}

}  // extern "C"
