// cvs_server.cpp - continuous-batching request loop of libcvsearch.
//
// Frames arrive (cvs_server_submit) while earlier frames are on the GPU.  A
// scheduler thread admits queued frames in arrival order whenever a slot (a
// context + stream) is free and the device arena has room for the frame and
// its maps; admitted frames are copied in and searched on their slot's stream,
// so several frames' copies and kernels overlap on the device.  Results stay
// resident in the arena until the client releases them.  All device memory is
// allocated at creation: admission never calls cudaMalloc.  Every host wait is
// bounded; no device-side wait exists.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "cvs_arena.h"
#include "cvs_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() {
    return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

cvs_status fail(cvs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    cvs::set_error_message(buf);
    return st;
}

struct Request {
    uint64_t id = 0;
    const uint8_t* host = nullptr;
    int32_t w = 0, h = 0;
    int64_t pitch = 0;
    int32_t state = CVS_REQ_QUEUED;
    int64_t off = -1;  // arena block: frame, then max_r, count, pmask
    int slot = -1;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    cvs_status err = CVS_OK;
    int64_t px() const { return (int64_t)w * h; }
    int64_t frame_bytes() const { return (px() * 3 + 255) / 256 * 256; }
    int64_t map_bytes() const { return px() * 9; }
};

struct Slot {
    cvs_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t req = 0;  // 0 = free
};

}  // namespace

struct cvs_server {
    cvs_server_config cfg{};
    std::vector<double> radii, angles;
    cvs_grid grid{};
    cvs_thresholds thr{};
    cvs_precision prec = CVS_PREC_FP32_RECHECK;
    unsigned char* arena_base = nullptr;
    cvs::Arena arena;
    cvs_lut* lut = nullptr;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> queue;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    std::vector<double> lat_ms;
    double t_first_submit = -1.0, t_last_done = 0.0;
    int64_t submitted = 0, completed = 0, failed = 0;
    cvs_status worker_err = CVS_OK;
};

namespace {

// Issue one admitted request on its slot: copy in, search (or look up), mark.
cvs_status issue(cvs_server* S, Slot& slot, Request& r) {
    unsigned char* base = S->arena_base + r.off;
    unsigned char* frame = base;
    float* max_r = reinterpret_cast<float*>(base + r.frame_bytes());
    int32_t* count = reinterpret_cast<int32_t*>(base + r.frame_bytes() + 4 * r.px());
    uint8_t* pmask = base + r.frame_bytes() + 8 * r.px();
    cudaError_t e = cudaMemcpy2DAsync(frame, (size_t)r.w * 3, r.host, (size_t)r.pitch,
                                      (size_t)r.w * 3, (size_t)r.h, cudaMemcpyHostToDevice, slot.st);
    if (e != cudaSuccess) return fail(CVS_ERR_CUDA, "frame copy: %s", cudaGetErrorString(e));
    cvs_image im{frame, r.w, r.h, (int64_t)r.w * 3};
    cvs_capacity_map m{max_r, count, pmask};
    cvs_status st = S->lut ? cvs_lut_lookup_images(S->lut, &im, 1, &m, slot.st)
                           : cvs_search_images(slot.ctx, &im, 1, &S->grid, &S->thr, S->prec, &m,
                                               slot.st);
    if (st != CVS_OK) return st;
    e = cudaEventRecord(slot.done, slot.st);
    if (e != cudaSuccess) return fail(CVS_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    return CVS_OK;
}

void worker_main(cvs_server* S) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progress = false;
        // completions
        for (size_t i = 0; i < S->slots.size(); ++i) {
            Slot& sl = S->slots[i];
            if (!sl.req) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            Request& r = S->reqs[sl.req];
            r.t_done = now_ms();
            if (q == cudaSuccess) {
                r.state = CVS_REQ_DONE;
                S->lat_ms.push_back(r.t_done - r.t_submit);
                ++S->completed;
                S->t_last_done = r.t_done;
            } else {
                r.state = CVS_REQ_FAILED;
                r.err = CVS_ERR_CUDA;
                ++S->failed;
            }
            sl.req = 0;
            progress = true;
        }
        // admissions, in arrival order
        while (!S->queue.empty()) {
            int free_slot = -1;
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].req) { free_slot = (int)i; break; }
            if (free_slot < 0) break;
            Request& r = S->reqs[S->queue.front()];
            const int64_t off = S->arena.alloc(r.frame_bytes() + r.map_bytes());
            if (off < 0) break;  // wait for releases
            S->queue.pop_front();
            r.off = off;
            r.slot = free_slot;
            r.t_start = now_ms();
            r.state = CVS_REQ_RUNNING;
            Slot& sl = S->slots[free_slot];
            sl.req = r.id;
            // the host-side staging of the frame copy can take milliseconds:
            // do not hold up submitters meanwhile (a RUNNING request cannot be
            // released, and map entries stay put while others are inserted)
            lk.unlock();
            const cvs_status st = issue(S, sl, r);
            lk.lock();
            if (st != CVS_OK) {
                // nothing of this request reached the device beyond what its
                // stream will finish; release it once the stream is idle
                cudaStreamSynchronize(sl.st);
                S->arena.release(r.off);
                r.off = -1;
                r.state = CVS_REQ_FAILED;
                r.err = st;
                ++S->failed;
                sl.req = 0;
            }
            progress = true;
        }
        if (progress) S->cv.notify_all();
        else S->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" {

cvs_status cvs_server_create(cvs_server** out, const cvs_server_config* cfg, const cvs_grid* grid,
                             const cvs_thresholds* thr, cvs_precision prec) {
    if (!out || !cfg || !grid || !thr) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->max_inflight > 16)
        return fail(CVS_ERR_INVALID_ARG, "max_inflight must be in [1, 16]");
    if (cfg->max_pixels < 1) return fail(CVS_ERR_INVALID_ARG, "max_pixels must be >= 1");
    if (cfg->mem_budget_bytes < cfg->max_pixels * 12 + 512)
        return fail(CVS_ERR_INVALID_ARG, "mem_budget_bytes cannot hold one frame of max_pixels");
    int32_t hi, lo;
    cvs_status st = cvs_signal_bounds(thr, &hi, &lo);
    if (st != CVS_OK) return st;
    if (!grid->radii || !grid->angles_deg || grid->n_radii <= 0 || grid->n_angles <= 0)
        return fail(CVS_ERR_INVALID_ARG, "empty or NULL grid");
    if (prec == CVS_PREC_FP32_RECHECK)
        for (int i = 0; i < grid->n_radii; ++i)
            if (grid->radii[i] > cvs::kFp32MaxRadius)
                return fail(CVS_ERR_INVALID_ARG,
                            "CVS_PREC_FP32_RECHECK is validated for radii up to %g: pass "
                            "CVS_PREC_FP64 for this grid", cvs::kFp32MaxRadius);
    cvs_server* S = new cvs_server();
    S->cfg = *cfg;
    S->radii.assign(grid->radii, grid->radii + grid->n_radii);
    S->angles.assign(grid->angles_deg, grid->angles_deg + grid->n_angles);
    S->grid = cvs_grid{S->radii.data(), grid->n_radii, S->angles.data(), grid->n_angles};
    S->thr = *thr;
    S->prec = prec;
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_base, (size_t)cfg->mem_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        return fail(e == cudaErrorMemoryAllocation ? CVS_ERR_NO_MEMORY : CVS_ERR_CUDA,
                    "server arena: %s", cudaGetErrorString(e));
    }
    S->arena.reset(cfg->mem_budget_bytes);
    S->slots.resize(cfg->max_inflight);
    st = CVS_OK;
    if (cfg->use_table) {
        cvs_ctx* c0 = nullptr;
        st = cvs_create(&c0, cfg->device, 0);
        if (st == CVS_OK) st = cvs_lut_build(c0, &S->grid, &S->thr, prec, &S->lut, nullptr);
        if (c0) cvs_destroy(c0);
    }
    for (size_t i = 0; i < S->slots.size() && st == CVS_OK; ++i) {
        Slot& sl = S->slots[i];
        if (!cfg->use_table) {
            st = cvs_create(&sl.ctx, cfg->device, 0);
            if (st == CVS_OK) st = cvs_reserve(sl.ctx, &S->grid, cfg->max_pixels, 1);
            if (st == CVS_OK) st = cvs::prepare_thresholds(sl.ctx, &S->thr);
            // leave room on every SM for the other slots' kernels
            const int per_sm = 5 / cfg->max_inflight;
            if (st == CVS_OK && cfg->max_inflight > 1)
                st = cvs_set_option(sl.ctx, "blocks_per_sm", per_sm < 1 ? 1 : per_sm);
            // de-duplicate per frame or not, fixed at creation (no table is
            // allocated while serving)
            if (st == CVS_OK) st = cvs_set_option(sl.ctx, "dedup", cfg->dedup ? 1 : 0);
        }
        if (st != CVS_OK) break;
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e != cudaSuccess) st = fail(CVS_ERR_CUDA, "slot: %s", cudaGetErrorString(e));
    }
    if (st != CVS_OK) {
        cvs_server_destroy(S);
        return st;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return CVS_OK;
}

void cvs_server_destroy(cvs_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->cfg.device);
    for (Slot& sl : S->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ctx) cvs_destroy(sl.ctx);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    if (S->lut) cvs_lut_destroy(S->lut);
    if (S->arena_base) cudaFree(S->arena_base);
    delete S;
}

cvs_status cvs_server_submit(cvs_server* S, const uint8_t* rgb_host, int32_t width,
                             int32_t height, int64_t pitch_bytes, uint64_t* ticket) {
    if (!S || !rgb_host || !ticket) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (width <= 0 || height <= 0 || pitch_bytes < 3LL * width)
        return fail(CVS_ERR_INVALID_ARG, "bad frame size or pitch");
    if ((int64_t)width * height > S->cfg.max_pixels)
        return fail(CVS_ERR_INVALID_ARG, "frame has %lld pixels, the server accepts %lld",
                    (long long)width * height, (long long)S->cfg.max_pixels);
    Request r;
    r.host = rgb_host;
    r.w = width;
    r.h = height;
    r.pitch = pitch_bytes;
    if (r.frame_bytes() + r.map_bytes() > S->arena.size())
        return fail(CVS_ERR_INVALID_ARG, "frame larger than the server's memory budget");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r.id = S->next_id++;
        r.t_submit = now_ms();
        if (S->t_first_submit < 0) S->t_first_submit = r.t_submit;
        S->reqs[r.id] = r;
        S->queue.push_back(r.id);
        ++S->submitted;
        *ticket = r.id;
    }
    S->cv.notify_all();
    return CVS_OK;
}

cvs_status cvs_server_state(cvs_server* S, uint64_t ticket, int32_t* state) {
    if (!S || !state) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    *state = it == S->reqs.end() ? CVS_REQ_UNKNOWN : it->second.state;
    return CVS_OK;
}

cvs_status cvs_server_wait(cvs_server* S, uint64_t ticket, int32_t timeout_ms) {
    if (!S) return fail(CVS_ERR_INVALID_ARG, "NULL server");
    if (timeout_ms < 0) return fail(CVS_ERR_INVALID_ARG, "timeout must be >= 0");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CVS_ERR_INVALID_ARG, "unknown ticket %llu",
                                         (unsigned long long)ticket);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    while (true) {
        it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(CVS_ERR_INVALID_ARG, "ticket released while waiting");
        if (it->second.state == CVS_REQ_DONE) return CVS_OK;
        if (it->second.state == CVS_REQ_FAILED)
            return fail(it->second.err == CVS_OK ? CVS_ERR_CUDA : it->second.err,
                        "request %llu failed", (unsigned long long)ticket);
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = S->reqs.find(ticket);
            if (it != S->reqs.end() && it->second.state == CVS_REQ_DONE) return CVS_OK;
            return fail(CVS_ERR_TIMEOUT, "request %llu not done after %d ms",
                        (unsigned long long)ticket, timeout_ms);
        }
    }
}

cvs_status cvs_server_result(cvs_server* S, uint64_t ticket, cvs_capacity_map* maps,
                             int32_t* width, int32_t* height) {
    if (!S || !maps) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CVS_ERR_INVALID_ARG, "unknown ticket");
    const Request& r = it->second;
    if (r.state != CVS_REQ_DONE) return fail(CVS_ERR_INVALID_ARG, "request not done");
    unsigned char* base = S->arena_base + r.off;
    maps->max_r = reinterpret_cast<float*>(base + r.frame_bytes());
    maps->count = reinterpret_cast<int32_t*>(base + r.frame_bytes() + 4 * r.px());
    maps->pmask = base + r.frame_bytes() + 8 * r.px();
    if (width) *width = r.w;
    if (height) *height = r.h;
    return CVS_OK;
}

cvs_status cvs_server_copy_result(cvs_server* S, uint64_t ticket, float* max_r_host,
                                  int32_t* count_host, uint8_t* pmask_host) {
    if (!S || !max_r_host || !count_host || !pmask_host)
        return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    cvs_capacity_map m{};
    int32_t w = 0, h = 0;
    cvs_status st = cvs_server_result(S, ticket, &m, &w, &h);
    if (st != CVS_OK) return st;
    const size_t px = (size_t)w * h;
    cudaError_t e = cudaSetDevice(S->cfg.device);
    if (e == cudaSuccess) e = cudaMemcpy(max_r_host, m.max_r, 4 * px, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(count_host, m.count, 4 * px, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(pmask_host, m.pmask, px, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(CVS_ERR_CUDA, "result copy: %s", cudaGetErrorString(e));
    return CVS_OK;
}

cvs_status cvs_server_release(cvs_server* S, uint64_t ticket) {
    if (!S) return fail(CVS_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(CVS_ERR_INVALID_ARG, "unknown ticket");
        Request& r = it->second;
        if (r.state == CVS_REQ_RUNNING)
            return fail(CVS_ERR_INVALID_ARG, "request still running; wait for it first");
        if (r.state == CVS_REQ_QUEUED) {
            S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), ticket), S->queue.end());
        }
        if (r.off >= 0) S->arena.release(r.off);
        S->reqs.erase(it);
    }
    S->cv.notify_all();
    return CVS_OK;
}

cvs_status cvs_server_get_stats(cvs_server* S, cvs_server_stats* out) {
    if (!S || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    cvs_server_stats s{};
    s.submitted = S->submitted;
    s.completed = S->completed;
    s.failed = S->failed;
    s.queued = (int64_t)S->queue.size();
    for (const Slot& sl : S->slots) s.inflight += sl.req ? 1 : 0;
    s.bytes_in_use = S->arena.in_use();
    s.peak_bytes_in_use = S->arena.peak();
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)(p * (double)(v.size() - 1) + 0.5);
            return v[i < v.size() ? i : v.size() - 1];
        };
        s.p50_ms = pct(0.50);
        s.p99_ms = pct(0.99);
        s.max_ms = v.back();
        double sum = 0.0;
        for (double x : v) sum += x;
        s.mean_ms = sum / (double)v.size();
        const double span = S->t_last_done - S->t_first_submit;
        s.frames_per_s = span > 0 ? (double)S->completed / (span / 1e3) : 0.0;
    }
    *out = s;
    return CVS_OK;
}

}  // extern "C"
