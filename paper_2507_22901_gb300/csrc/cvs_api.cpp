// cvs_api.cpp - host side of libcvsearch: the C ABI declared in
// include/cvsearch.h.  Validates arguments, owns the context's scratch memory
// and grid tables, and launches the kernels of cvs_kernels.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "cvs_internal.h"

using namespace cvs;

namespace {

thread_local std::string g_err;

cvs_status fail(cvs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CVS_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? CVS_ERR_NO_MEMORY : CVS_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

constexpr int32_t kMaxGrid = 8192;  // shared-memory tables: 8 B per radius, 16 B per angle slot

}  // namespace

void cvs::set_error_message(const char* msg) { g_err = msg; }

int cvs::auto_kchunk(int num_sms, int64_t n_targets, int K, int H) {
    // aim for >= 32 work items per SM warp-slot group, but >= 2 warp iterations per item
    const int64_t want_items = (int64_t)num_sms * 512;
    int64_t n_kc = (want_items + n_targets - 1) / (n_targets > 0 ? n_targets : 1);
    if (n_kc < 1) n_kc = 1;
    if (n_kc > K) n_kc = K;
    int kchunk = (int)((K + n_kc - 1) / n_kc);
    const int min_k = (64 + H - 1) / H;
    if (kchunk < min_k) kchunk = min_k < K ? min_k : K;
    return kchunk;
}

int cvs::fold_by_180(const double* s, const double* c, int N) {
    if (N % 2) return 0;
    for (int m = 0; m < N / 2; ++m)
        if (!(s[m + N / 2] == -s[m] && c[m + N / 2] == -c[m])) return 0;
    return 1;
}

struct cvs_ctx {
    int device = 0;
    int num_sms = 0;
    // device memory the context owns (scratch, tables, graph copies), with
    // its size, counted against the budget given to cvs_create (0 = none)
    size_t budget = 0, in_use = 0;
    std::unordered_map<void*, size_t> owned;
    cudaStream_t own = nullptr;  // stream of the synchronous entry points
    // grid cache
    std::vector<double> radii, angles;
    GridDev grid;
    double* d_angles = nullptr;
    int64_t cap_grid = 0;
    int* d_status = nullptr;
    // per-target scratch
    TargetF32* tf = nullptr;
    TargetF64* td = nullptr;
    Acc* acc = nullptr;
    int64_t cap_tf = 0, cap_td = 0, cap_acc = 0;
    long long* qkey = nullptr;
    unsigned long long* counters = nullptr;  // kNumCounters: work, flagged, rechecked, n_out, skipped
    unsigned long long* h_counters = nullptr;  // pinned copy
    // pair lists: records of cvs_search_color; per work item of a batch its
    // passing-slot bitmap, count and scan base; per tile of the scan its base
    cvs_pair* compact = nullptr;
    int64_t cap_compact = 0;
    uint32_t* d_bits = nullptr;
    int64_t cap_bits = 0;
    uint32_t* d_icount = nullptr;
    int64_t cap_icount = 0;
    int64_t* d_within = nullptr;
    int64_t cap_within = 0;
    int64_t* d_tiles = nullptr;
    int64_t cap_tiles = 0;
    int64_t list_batch_items = int64_t(1) << 22;  // most work items per batch
    // images
    ImageDesc* d_imgs = nullptr;
    int64_t cap_imgs = 0;
    // host-buffer entry point
    uint8_t* d_in = nullptr;
    float* d_maxr = nullptr;
    int32_t* d_count = nullptr;
    uint8_t* d_pmask = nullptr;
    int64_t cap_in = 0, cap_maxr = 0, cap_count = 0, cap_pmask = 0;
    uint8_t* d_rgb1 = nullptr;  // 3 bytes for cvs_search_color
    // probe
    unsigned int* d_probe = nullptr;
    // options
    LaunchShape shape;
    double window = 2e-3;  // FP32 flag window W in code units
    // last call
    cvs_stats last{};
    bool last_pending = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the search kernel
    cudaEvent_t ev_mid = nullptr;  // after the angle-ranges pass (first chunk)
    bool last_arcs = false;        // the last search took the angle ranges
    // autotuning: best launch shape per (grid, precision, modes, size bucket)
    int autotune = 0;
    std::map<std::array<int64_t, 7>, LaunchShape> tuned;
    Acc* acc_tune = nullptr;
    int64_t cap_acc_tune = 0;
    // the FP32 search walks per-radius angle ranges where the grid allows:
    // 0 never, 1 always, 2 where a probe of the first call per grid and
    // thresholds finds they list well under the slots of the plain walk
    int angle_ranges = 2;
    uint2* arc_ranges = nullptr;  // scratch of the angle ranges
    int64_t cap_arc = 0;
    unsigned long long* d_arc_probe = nullptr;
    unsigned long long* h_arc_probe = nullptr;
    std::map<std::array<int64_t, 6>, bool> arc_choice;
    int search_kind = 0;  // kind of the current call, part of the choice's key
    // per-batch colour de-duplication of the image search (option "dedup":
    // 0 never, 1 always, 2 automatic)
    int dedup = 2;
    uint8_t* d_present = nullptr;   // 2^24 bytes
    int32_t* d_index = nullptr;     // 2^24 colour -> distinct-colour index
    uint8_t* d_unique = nullptr;    // 3 x 2^24 distinct colours
    int* d_scan = nullptr;          // 1024 block sums + the distinct count
    int* h_unique = nullptr;        // pinned copy of the distinct count
    // pair lists of many colours: per-colour offsets into the caller's output
    int64_t* d_offs = nullptr;
    int64_t cap_offs = 0;
    // L* of all 2^24 colours, built by the first call with a luminance limit
    double* ltab = nullptr;
    // 1: CVS_PREC_FP32_RECHECK on a grid with a radius above kFp32MaxRadius
    // runs in FP64; 0 (default): such a call is refused
    int fp64_fallback = 0;
    // embedding: radius indices sorted by (radius value, index), K entries
    int32_t* d_order = nullptr;
    // multi-threshold search: n x n_thr accumulators
    Acc* acc_multi = nullptr;
    int64_t cap_acc_multi = 0;
    unsigned long long* tune_counters = nullptr;
    // CUDA graphs: one captured setup+search+finalize sequence per input signature
    int use_graphs = 0;
    struct GraphEntry {
        std::vector<uint64_t> key;
        cudaGraphExec_t exec = nullptr;
        ImageDesc* d_imgs = nullptr;
        uint64_t last_use = 0;
    };
    std::vector<GraphEntry> graphs;
    uint64_t graph_clock = 0;
    uint64_t grid_gen = 0, scratch_gen = 0;
    cudaStream_t cap = nullptr;  // capture stream
    int64_t graph_launches = 0;
};

namespace {

// Allocate `bytes` of device memory owned by the context, within its budget.
cvs_status ctx_alloc(cvs_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (c->budget && c->in_use + bytes > c->budget)
        return fail(CVS_ERR_NO_MEMORY,
                    "context memory budget of %zu bytes exceeded: %zu in use, %zu more needed",
                    c->budget, c->in_use, bytes);
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CVS_ERR_NO_MEMORY : CVS_ERR_CUDA,
                    "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->owned[*p] = bytes;
    c->in_use += bytes;
    return CVS_OK;
}

template <class T>
cvs_status ctx_alloc(cvs_ctx* c, T** p, size_t bytes) {
    void* v = nullptr;
    const cvs_status st = ctx_alloc(c, &v, bytes);
    *p = static_cast<T*>(v);
    return st;
}

// Release memory from ctx_alloc (NULL is ignored).
void ctx_free(cvs_ctx* c, void* p) {
    if (!p) return;
    auto it = c->owned.find(p);
    if (it != c->owned.end()) {
        c->in_use -= it->second;
        c->owned.erase(it);
    }
    cudaFree(p);
}

// Make *p hold at least `need` elements (contents are not kept).
template <class T>
cvs_status grow(cvs_ctx* c, T** p, int64_t* cap, int64_t need) {
    if (*cap >= need && *p) return CVS_OK;
    ctx_free(c, *p);
    *p = nullptr;
    *cap = 0;
    const int64_t n = need < 1 ? 1 : need;
    const cvs_status st = ctx_alloc(c, p, (size_t)n * sizeof(T));
    if (st == CVS_OK) *cap = n;
    return st;
}

#define CVS_TRY(call)                        \
    do {                                     \
        const cvs_status s_ = (call);        \
        if (s_ != CVS_OK) return s_;         \
    } while (0)

cvs_status set_device(cvs_ctx* c) {
    CVS_CUDA(cudaSetDevice(c->device));
    return CVS_OK;
}

cvs_status check_thresholds(const cvs_thresholds* t) {
    if (!t) return fail(CVS_ERR_INVALID_ARG, "thresholds pointer is NULL");
    if (!std::isfinite(t->v_th) || t->v_th < 0.0)
        return fail(CVS_ERR_INVALID_ARG, "v_th must be finite and >= 0 (got %g)", t->v_th);
    if (!(t->r_novib > 0.0 && t->r_novib <= 1.0))
        return fail(CVS_ERR_INVALID_ARG, "r_novib must be in (0, 1] (got %g)", t->r_novib);
    if (t->pattern_mask > 0x7Fu)
        return fail(CVS_ERR_INVALID_ARG, "pattern_mask has bits above the 7 patterns (0x%x)",
                    t->pattern_mask);
    if (t->gamut_mode != 0 && t->gamut_mode != 1)
        return fail(CVS_ERR_INVALID_ARG, "gamut_mode must be 0 (reject) or 1 (clip)");
    if (std::isnan(t->max_dl) || t->max_dl < 0.0)
        return fail(CVS_ERR_INVALID_ARG,
                    "max_dl must be 0 or +inf (no limit) or a positive limit (got %g)", t->max_dl);
    return CVS_OK;
}

// The luminance limit of a threshold set is on for a positive, finite max_dl.
bool dl_on(const cvs_thresholds* t) { return t->max_dl > 0.0 && std::isfinite(t->max_dl); }

// The L* table of all 2^24 colours that the luminance limit reads, built once
// (synchronously, outside any capture) by the first call that needs it.
cvs_status ensure_ltab(cvs_ctx* c, const cvs_thresholds* t) {
    if (!dl_on(t) || c->ltab) return CVS_OK;
    CVS_TRY(ctx_alloc(c, &c->ltab, sizeof(double) << 24));
    CVS_CUDA(launch_l_table(c->ltab, c->own));
    CVS_CUDA(cudaStreamSynchronize(c->own));
    return CVS_OK;
}

}  // namespace

cvs_status cvs::prepare_thresholds(cvs_ctx* c, const cvs_thresholds* t) {
    cvs_status st = check_thresholds(t);
    if (st == CVS_OK) st = set_device(c);
    if (st == CVS_OK) st = ensure_ltab(c, t);
    return st;
}

namespace {

cvs_status check_grid(const cvs_grid* g) {
    if (!g) return fail(CVS_ERR_INVALID_ARG, "grid pointer is NULL");
    if (!g->radii || !g->angles_deg) return fail(CVS_ERR_INVALID_ARG, "grid arrays are NULL");
    if (g->n_radii <= 0 || g->n_radii > kMaxGrid)
        return fail(CVS_ERR_INVALID_ARG, "n_radii must be in [1, %d] (got %d)", kMaxGrid, g->n_radii);
    if (g->n_angles <= 0 || g->n_angles > kMaxGrid)
        return fail(CVS_ERR_INVALID_ARG, "n_angles must be in [1, %d] (got %d)", kMaxGrid,
                    g->n_angles);
    for (int i = 0; i < g->n_radii; ++i)
        if (!std::isfinite(g->radii[i]) || g->radii[i] < 0.0 || g->radii[i] > kMaxRadius)
            return fail(CVS_ERR_INVALID_ARG, "radius %d must be in [0, %g] (got %g)", i, kMaxRadius,
                        g->radii[i]);
    for (int i = 0; i < g->n_angles; ++i)
        if (!std::isfinite(g->angles_deg[i]))
            return fail(CVS_ERR_INVALID_ARG, "angle %d is not finite", i);
    return CVS_OK;
}

// Upload the grid and build its tables on the device (cached by content).
cvs_status ensure_grid(cvs_ctx* c, const cvs_grid* g) {
    if (c->grid.K == g->n_radii && c->grid.N == g->n_angles &&
        std::memcmp(c->radii.data(), g->radii, sizeof(double) * g->n_radii) == 0 &&
        std::memcmp(c->angles.data(), g->angles_deg, sizeof(double) * g->n_angles) == 0)
        return CVS_OK;
    GridDev& d = c->grid;
    const int K = g->n_radii, N = g->n_angles;
    // earlier asynchronous searches may still read the old tables
    CVS_CUDA(cudaDeviceSynchronize());
    d.K = 0;  // invalid until complete
    if (c->cap_grid < kMaxGrid) {
        CVS_TRY(ctx_alloc(c, &d.r32, sizeof(float) * kMaxGrid));
        CVS_TRY(ctx_alloc(c, &d.sc32, sizeof(float2) * kMaxGrid));
        CVS_TRY(ctx_alloc(c, &d.r64, sizeof(double) * kMaxGrid));
        CVS_TRY(ctx_alloc(c, &d.s64, sizeof(double) * kMaxGrid));
        CVS_TRY(ctx_alloc(c, &d.c64, sizeof(double) * kMaxGrid));
        CVS_TRY(ctx_alloc(c, &c->d_angles, sizeof(double) * kMaxGrid));
        CVS_TRY(ctx_alloc(c, &c->d_order, sizeof(int32_t) * kMaxGrid));
        c->cap_grid = kMaxGrid;
    }
    std::vector<float> r32(K);
    double rmax = 0.0;
    for (int i = 0; i < K; ++i) {
        r32[i] = (float)g->radii[i];
        if (g->radii[i] > rmax) rmax = g->radii[i];
    }
    std::vector<int32_t> order(K);
    for (int i = 0; i < K; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [g](int32_t x, int32_t y) { return g->radii[x] < g->radii[y]; });
    cudaStream_t st = c->own;
    CVS_CUDA(cudaMemcpyAsync(c->d_order, order.data(), sizeof(int32_t) * K,
                             cudaMemcpyHostToDevice, st));
    CVS_CUDA(cudaMemcpyAsync(d.r64, g->radii, sizeof(double) * K, cudaMemcpyHostToDevice, st));
    CVS_CUDA(cudaMemcpyAsync(d.r32, r32.data(), sizeof(float) * K, cudaMemcpyHostToDevice, st));
    CVS_CUDA(cudaMemcpyAsync(c->d_angles, g->angles_deg, sizeof(double) * N,
                             cudaMemcpyHostToDevice, st));
    CVS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
    CVS_CUDA(launch_trig_table(c->d_angles, N, d.s64, d.c64, d.sc32, c->d_status, st));
    std::vector<double> s(N), co(N);
    int status = 0;
    CVS_CUDA(cudaMemcpyAsync(s.data(), d.s64, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CVS_CUDA(cudaMemcpyAsync(co.data(), d.c64, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CVS_CUDA(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CVS_CUDA(cudaStreamSynchronize(st));
    if (status) return fail(CVS_ERR_NUMERIC, "an angle's sine could not be certified");
    const int sym = fold_by_180(s.data(), co.data(), N);
    d.sym = sym;
    d.H = sym ? N / 2 : N;
    // Angle ranges need slot h at angle angles[0] + h * 360 / N, h < N / 2,
    // to within 1e-6 degrees (the ranges carry a margin of 2e-4 rad).
    int even = sym;
    const double step = 360.0 / N;
    for (int m = 0; even && m < N / 2; ++m) {
        const double want = g->angles_deg[0] + m * step;
        if (!(std::fabs(g->angles_deg[m] - want) <= 1e-6)) even = 0;
    }
    d.arcs_ok = even;
    // The first angle reduced to [0, 360) in double before it is rounded to
    // FP32 radians: fmod is exact, so a large offset (say 1e6 + 0.5 degrees)
    // costs no more than the final FP32 rounding (< 4e-7 rad).
    double th0_deg = std::fmod(g->angles_deg[0], 360.0);
    if (th0_deg < 0.0) th0_deg += 360.0;
    d.th0 = (float)(th0_deg * (3.14159265358979323846 / 180.0));
    d.inv_step = even ? (float)(N / (2.0 * 3.14159265358979323846)) : 0.0f;
    d.arcs = d.arcs_ok && c->angle_ranges;
    d.N = N;
    d.rmax = rmax;
    c->radii.assign(g->radii, g->radii + K);
    c->angles.assign(g->angles_deg, g->angles_deg + N);
    d.K = K;
    ++c->grid_gen;
    return CVS_OK;
}

void drop_graphs(cvs_ctx* c);

cvs_status ensure_arc_scratch(cvs_ctx* c, int64_t n);

// Tables of the per-batch colour de-duplication (option "dedup"): presence
// map and index of all 2^24 colours, the distinct colours, scan sums (each
// allocated if missing, so a refused allocation can be retried).
cvs_status ensure_dedup(cvs_ctx* c) {
    constexpr size_t kColours = size_t(1) << 24;
    if (!c->d_present) CVS_TRY(ctx_alloc(c, &c->d_present, kColours));
    if (!c->d_index) CVS_TRY(ctx_alloc(c, &c->d_index, sizeof(int32_t) * kColours));
    if (!c->d_unique) CVS_TRY(ctx_alloc(c, &c->d_unique, 3 * kColours));
    if (!c->d_scan) CVS_TRY(ctx_alloc(c, &c->d_scan, sizeof(int) * 1025));
    if (!c->h_unique) CVS_CUDA(cudaMallocHost(&c->h_unique, sizeof(int)));
    return CVS_OK;
}

// Frees the de-duplication tables (after a refused allocation of the automatic
// mode, so that a partial set does not hold budget the per-pixel search needs).
void drop_dedup(cvs_ctx* c) {
    ctx_free(c, c->d_present);
    ctx_free(c, c->d_index);
    ctx_free(c, c->d_unique);
    ctx_free(c, c->d_scan);
    c->d_present = nullptr;
    c->d_index = nullptr;
    c->d_unique = nullptr;
    c->d_scan = nullptr;
}

// Option "dedup" = 2 (the default): batches of at least this many pixels are
// searched once per distinct colour, when CUDA graphs are off and the tables
// fit the context's memory budget.
constexpr int64_t kDedupAutoPixels = int64_t(1) << 20;

// The FP32 path's error bound is validated for radii up to kFp32MaxRadius:
// on a grid with a larger radius an FP32 request is refused, or (option
// "fp64_fallback") turned into FP64, which cvs_stats.precision reports.
cvs_status resolve_precision(cvs_ctx* c, cvs_precision* prec) {
    if (*prec != CVS_PREC_FP32_RECHECK || c->grid.rmax <= kFp32MaxRadius) return CVS_OK;
    if (!c->fp64_fallback)
        return fail(CVS_ERR_INVALID_ARG,
                    "CVS_PREC_FP32_RECHECK is validated for radii up to %g and the grid has %g: "
                    "pass CVS_PREC_FP64 (about 100x slower), or set option \"fp64_fallback\" to "
                    "1 to have such grids run in FP64", kFp32MaxRadius, c->grid.rmax);
    *prec = CVS_PREC_FP64;
    return CVS_OK;
}

cvs_status ensure_targets(cvs_ctx* c, int64_t n) {
    if (c->cap_tf < n || c->cap_td < n || c->cap_acc < n) {
        drop_graphs(c);  // captured graphs point at the buffers about to be replaced
        ++c->scratch_gen;
    }
    if (c->cap_tf < n) {
        ctx_free(c, c->tf);
        c->tf = nullptr;
        c->cap_tf = 0;
        CVS_TRY(ctx_alloc(c, &c->tf, target_f32_size() * (size_t)n));
        c->cap_tf = n;
    }
    if (c->cap_td < n) {
        ctx_free(c, c->td);
        c->td = nullptr;
        c->cap_td = 0;
        CVS_TRY(ctx_alloc(c, &c->td, target_f64_size() * (size_t)n));
        c->cap_td = n;
    }
    CVS_TRY(grow(c, &c->acc, &c->cap_acc, n));
    return ensure_arc_scratch(c, n);  // before any capture can need it
}

void thresholds_to_int(const cvs_thresholds* t, int32_t* hi_min, int32_t* lo_max) {
    // high: d > v_th  <=>  d >= floor(v_th) + 1
    const double fl = std::floor(t->v_th);
    *hi_min = fl >= 255.0 ? 256 : (int32_t)fl + 1;
    // low: d < v_th * r_novib (exact product)  <=>  d <= ceil(product) - 1
    const double p = t->v_th * t->r_novib;
    const double e = std::fma(t->v_th, t->r_novib, -p);  // product = p + e exactly
    double ce = std::ceil(p);
    if (ce == p && e > 0.0) ce += 1.0;
    *lo_max = ce > 256.0 ? 255 : (int32_t)ce - 1;
}

int choose_kchunk(const cvs_ctx* c, int64_t n_targets, int K, int H) {
    if (c->shape.kchunk > 0) return c->shape.kchunk < K ? c->shape.kchunk : K;
    return auto_kchunk(c->num_sms, n_targets, K, H);
}

std::array<int64_t, 7> tune_key(const cvs_ctx* c, int64_t n, int prec, int clip, int list) {
    int64_t bucket = 0;
    while ((int64_t(1) << (bucket + 1)) <= n) ++bucket;
    return {c->grid.K, c->grid.H, c->grid.sym, prec, clip, list, bucket};
}

// Time candidate launch shapes of the search on (a prefix of) the prepared
// targets and return the fastest.  Accumulates into a separate buffer, so the
// caller's accumulators are untouched.  Synchronous on `st`.
cvs_status tune_shape(cvs_ctx* c, const SearchArgs& base, cudaStream_t st, LaunchShape* best,
                      double* best_ms) {
    const int K = c->grid.K, H = c->grid.H;
    // sample: at most ~3e10 candidates per timed launch
    int64_t n = base.n_targets;
    const int64_t per_target = (int64_t)K * H * (c->grid.sym ? 2 : 1);
    const int64_t cap = (int64_t)3e10 / (per_target > 0 ? per_target : 1);
    if (n > cap) n = cap < 1 ? 1 : cap;
    CVS_TRY(grow(c, &c->acc_tune, &c->cap_acc_tune, n));
    if (!c->tune_counters)
        CVS_TRY(ctx_alloc(c, &c->tune_counters, kNumCounters * sizeof(unsigned long long)));
    std::vector<LaunchShape> cand;
    const int auto_k = choose_kchunk(c, n, K, H);
    const int min_k = (64 + H - 1) / H;
    for (int block : {64, kSearchBlock}) {
        std::vector<int> ks = {auto_k, K};
        for (int div = 2; div <= 64; div *= 2) {
            const int kc = (K + div - 1) / div;
            if (kc >= min_k && kc >= 1) ks.push_back(kc);
        }
        std::vector<int> seen;
        for (int kc : ks) {
            bool dup = false;
            for (int v : seen) dup |= v == kc;
            if (dup) continue;
            seen.push_back(kc);
            LaunchShape sh;
            sh.block = block;
            sh.blocks_per_sm = 0;
            sh.kchunk = kc;
            cand.push_back(sh);
        }
    }
    cudaEvent_t e0, e1;
    CVS_CUDA(cudaEventCreate(&e0));
    CVS_CUDA(cudaEventCreate(&e1));
    *best_ms = 1e300;
    cvs_status status = CVS_OK;
    for (const LaunchShape& sh : cand) {
        SearchArgs a = base;
        a.n_targets = n;
        a.acc = c->acc_tune;
        a.work_counter = c->tune_counters;
        a.stats = c->tune_counters + 1;
        a.list_mode = 0;
        a.shape = sh;
        double ms_min = 1e300;
        for (int rep = 0; rep < 3 && status == CVS_OK; ++rep) {
            cudaError_t e = cudaMemsetAsync(c->tune_counters, 0, kNumCounters * sizeof(unsigned long long), st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch_search(a, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) status = fail(CVS_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
            if (rep > 0 && ms < ms_min) ms_min = ms;  // first run warms up
        }
        if (status != CVS_OK) break;
        if (ms_min < *best_ms) {
            *best_ms = ms_min;
            *best = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}

// Entries of angle-range scratch a search of n targets uses (one chunk).
int64_t arc_entries(const cvs_ctx* c, int64_t n) {
    const int64_t K = c->grid.K > 0 ? c->grid.K : 1;
    const int64_t per_chunk = kArcScratchEntries / K > 0 ? kArcScratchEntries / K : 1;
    return (n < per_chunk ? (n > 0 ? n : 1) : per_chunk) * K;
}

cvs_status ensure_arc_scratch(cvs_ctx* c, int64_t n) {
    if (!c->grid.arcs) return CVS_OK;
    if (!c->d_arc_probe) {  // the probe's counts (allocated with the scratch, ahead of any search)
        CVS_TRY(ctx_alloc(c, &c->d_arc_probe, 2 * sizeof(unsigned long long)));
        CVS_CUDA(cudaMallocHost(&c->h_arc_probe, 2 * sizeof(unsigned long long)));
    }
    const int64_t need = arc_entries(c, n);
    if (c->cap_arc >= need) return CVS_OK;
    drop_graphs(c);  // captured graphs point at the buffer about to be replaced
    ctx_free(c, c->arc_ranges);
    c->arc_ranges = nullptr;
    c->cap_arc = 0;
    CVS_TRY(ctx_alloc(c, &c->arc_ranges, sizeof(uint2) * (size_t)need));
    c->cap_arc = need;
    return CVS_OK;
}

// Angle ranges pay where they list well under the slots a plain walk searches
// (the walk over a list costs about a fifth more per slot, plus the ranges
// pass): measure both counts on targets spread evenly over the call,
// synchronously.
constexpr int64_t kArcProbeTargets = 4096;
constexpr double kArcProbeRatio = 0.6;

cvs_status arc_probe(cvs_ctx* c, const SearchArgs& a, int64_t n, cudaStream_t st,
                     std::map<std::array<int64_t, 6>, bool>::iterator* it,
                     const std::array<int64_t, 6>& key) {
    int64_t nt = n < kArcProbeTargets ? n : kArcProbeTargets;
    if (nt * c->grid.K > a.arc_cap) nt = a.arc_cap / c->grid.K;
    const int64_t stride = nt > 0 ? n / nt : 1;  // evenly over the call's targets
    CVS_CUDA(launch_arc_probe(a, nt, stride, c->d_arc_probe, st));
    CVS_CUDA(cudaMemcpyAsync(c->h_arc_probe, c->d_arc_probe, 2 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, st));
    CVS_CUDA(cudaStreamSynchronize(st));
    const double covered = (double)c->h_arc_probe[0], plain = (double)c->h_arc_probe[1];
    *it = c->arc_choice.emplace(key, covered < kArcProbeRatio * plain).first;
    return CVS_OK;
}

// The angle-range fields of a search of n targets: the scratch (grown unless
// inside a capture, where the plain walk runs instead) and, with option
// angle_ranges = 2, the probe's choice for this grid, thresholds and kind of
// call (probed once, synchronously, outside captures).
// With the automatic choice, a call of fewer (target, radius) pairs than
// this keeps the plain walk: on work that does not fill the GPU the range
// pass and its extra launches cost more than they save (the paper's Table 1
// experiment, 9 colours x 61 radii under 12 sets: 58 us on the plain walk, 77
// us with the ranges).
constexpr int64_t kArcMinPairs = int64_t(1) << 13;

cvs_status prepare_arcs(cvs_ctx* c, SearchArgs& a, int64_t n, cvs_precision prec, int list_mode,
                        cudaStream_t st, bool capturing) {
    if (c->angle_ranges == 2 && n * (int64_t)c->grid.K < kArcMinPairs) a.grid.arcs = 0;
    if (a.grid.arcs && prec == CVS_PREC_FP32_RECHECK) {
        const int64_t need = arc_entries(c, n);
        if (c->cap_arc < need && !capturing) {
            cvs_status as = ensure_arc_scratch(c, n);
            if (as != CVS_OK) return as;
        }
        if (c->cap_arc < need) a.grid.arcs = 0;  // (inside a capture) the plain walk
        a.arc_ranges = c->arc_ranges;
        a.arc_cap = c->cap_arc;
        if (a.grid.arcs && !a.clip && c->angle_ranges == 2) {
            // per kind of call too: colours, images and the all-colour table differ
            const std::array<int64_t, 6> key = {c->grid_gen, a.hi_min, a.lo_max, a.mask2,
                                                (int64_t)list_mode, c->search_kind};
            auto it = c->arc_choice.find(key);
            if (it == c->arc_choice.end() && !capturing) {
                cvs_status ps = arc_probe(c, a, n, st, &it, key);
                if (ps != CVS_OK) return ps;
            }
            if (it != c->arc_choice.end() && !it->second) a.grid.arcs = 0;
        }
    }
    a.num_sms = c->num_sms;
    return CVS_OK;
}

// The probe's key for the multi-threshold search (in place of a list mode).
constexpr int kMultiArcKey = 2;

// Where a pair-list search (list mode) leaves its work items' bitmaps and
// counts, and the radii per work item fixed for the whole call.
struct ListOut {
    uint32_t* item_bits = nullptr;
    int item_words = 0;
    uint32_t* item_count = nullptr;
    int kchunk = 1;
};

cvs_status run_search(cvs_ctx* c, int64_t n, const cvs_thresholds* thr, cvs_precision prec,
                      int list_mode, uint32_t target_id, cudaStream_t st, bool capturing = false,
                      const ListOut* lo = nullptr) {
    SearchArgs a{};
    a.tf = c->tf;
    a.td = c->td;
    a.acc = c->acc;
    a.n_targets = n;
    a.grid = c->grid;
    a.qkey = c->qkey;
    thresholds_to_int(thr, &a.hi_min, &a.lo_max);
    a.mask2 = thr->pattern_mask << 1;
    a.clip = thr->gamut_mode;
    a.half_w = (float)(0.5 - c->window);
    a.prec = (int32_t)prec;
    a.list_mode = list_mode;
    a.target_id = target_id;
    if (list_mode) {
        a.item_bits = lo->item_bits;
        a.item_words = lo->item_words;
        a.item_count = lo->item_count;
        a.item0 = 0;
    }
    a.ltab = dl_on(thr) ? c->ltab : nullptr;
    a.max_dl = thr->max_dl;
    a.work_counter = c->counters;
    a.stats = c->counters + 1;
    a.shape = c->shape;
    a.shape.kchunk = choose_kchunk(c, n, c->grid.K, c->grid.H);
    a.num_sms = c->num_sms;
    {
        cvs_status as = prepare_arcs(c, a, n, prec, list_mode, st, capturing);
        if (as != CVS_OK) return as;
    }
    // a tuned shape applies when the caller has not fixed the shape by hand
    if (c->shape.kchunk == 0 && c->shape.blocks_per_sm == 0 && c->shape.block == kSearchBlock) {
        const auto key = tune_key(c, n, (int)prec, a.clip, list_mode);
        auto it = c->tuned.find(key);
        if (it == c->tuned.end() && c->autotune && !capturing && !list_mode) {
            LaunchShape best;
            double ms = 0.0;
            cvs_status ts = tune_shape(c, a, st, &best, &ms);
            if (ts != CVS_OK) return ts;
            it = c->tuned.emplace(key, best).first;
        }
        if (it != c->tuned.end()) a.shape = it->second;
    }
    if (list_mode) a.shape.kchunk = lo->kchunk;
    const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    CVS_CUDA(cudaMemsetAsync(c->counters, 0, kNumCounters * sizeof(unsigned long long), st));
    a.ev_ranges = c->ev_mid;
    a.ev_flags = ev_flags;
    c->last_arcs = a.grid.arcs && !a.clip && prec == CVS_PREC_FP32_RECHECK && a.arc_ranges &&
                   a.arc_cap >= a.grid.K;
    CVS_CUDA(cudaEventRecordWithFlags(c->ev0, st, ev_flags));
    CVS_CUDA(launch_search(a, st));
    CVS_CUDA(cudaEventRecordWithFlags(c->ev1, st, ev_flags));
    CVS_CUDA(cudaMemcpyAsync(c->h_counters, c->counters, kNumCounters * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, st));
    cvs_stats& s = c->last;
    s = cvs_stats{};
    s.targets = n;
    s.candidates = n * (int64_t)c->grid.K * c->grid.N;
    s.colors_fp32 = prec == CVS_PREC_FP64 ? 0 : s.candidates;
    s.symmetric = c->grid.sym;
    s.precision = (int32_t)prec;
    c->last_pending = true;
    return CVS_OK;
}

void drop_graphs(cvs_ctx* c) {
    for (auto& g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        ctx_free(c, g.d_imgs);
    }
    c->graphs.clear();
}

uint64_t dbits(double x) {
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
}

// Launch a captured graph for `key` on `st`, capturing it first with
// `enqueue(stream)` on the context's capture stream if it is not cached.
template <class F>
cvs_status graph_launch(cvs_ctx* c, std::vector<uint64_t> key, cudaStream_t st, F enqueue,
                        const std::vector<ImageDesc>* imgs = nullptr) {
    key.push_back(c->grid_gen);
    key.push_back(c->scratch_gen);
    cvs_ctx::GraphEntry* hit = nullptr;
    for (auto& g : c->graphs)
        if (g.key == key) hit = &g;
    if (!hit) {
        if (c->graphs.size() >= 8) {  // evict the least recently used
            size_t lru = 0;
            for (size_t i = 1; i < c->graphs.size(); ++i)
                if (c->graphs[i].last_use < c->graphs[lru].last_use) lru = i;
            if (c->graphs[lru].exec) cudaGraphExecDestroy(c->graphs[lru].exec);
            ctx_free(c, c->graphs[lru].d_imgs);
            c->graphs.erase(c->graphs.begin() + lru);
        }
        cvs_ctx::GraphEntry e;
        e.key = key;
        if (imgs) {  // the graph's own copy of the image table
            CVS_TRY(ctx_alloc(c, &e.d_imgs, sizeof(ImageDesc) * imgs->size()));
            CVS_CUDA(cudaMemcpy(e.d_imgs, imgs->data(), sizeof(ImageDesc) * imgs->size(),
                                cudaMemcpyHostToDevice));
        }
        CVS_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        cvs_status est = enqueue(c->cap, e.d_imgs);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(c->cap, &graph);
        if (est != CVS_OK) {
            if (graph) cudaGraphDestroy(graph);
            ctx_free(c, e.d_imgs);
            return est;
        }
        if (ce != cudaSuccess) {
            ctx_free(c, e.d_imgs);
            return fail(CVS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            ctx_free(c, e.d_imgs);
            return fail(CVS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        }
        c->graphs.push_back(e);
        hit = &c->graphs.back();
    }
    hit->last_use = ++c->graph_clock;
    CVS_CUDA(cudaGraphLaunch(hit->exec, st));
    ++c->graph_launches;
    return CVS_OK;
}

void collect_stats(cvs_ctx* c) {
    if (!c->last_pending) return;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->last.search_ms = ms;
    c->last.ranges_ms = 0.0;
    if (c->last_arcs && cudaEventElapsedTime(&ms, c->ev0, c->ev_mid) == cudaSuccess)
        c->last.ranges_ms = ms;
    const int f = c->grid.sym ? 2 : 1;
    c->last.flagged = (int64_t)c->h_counters[1] * f;
    c->last.rechecked = (int64_t)c->h_counters[2] * f;
    c->last.skipped = (int64_t)c->h_counters[4] * f;
    c->last.pruned = (int64_t)c->h_counters[5] * f;
    c->last_pending = false;
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

const char* cvs_last_error(void) { return g_err.c_str(); }

const char* cvs_version(void) { return "0.1.0"; }

cvs_status cvs_create(cvs_ctx** out, int device, size_t mem_budget_bytes) {
    if (!out) return fail(CVS_ERR_INVALID_ARG, "ctx output pointer is NULL");
    *out = nullptr;
    int ndev = 0;
    CVS_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev)
        return fail(CVS_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, ndev);
    cvs_ctx* c = new cvs_ctx();
    c->device = device;
    c->budget = mem_budget_bytes;
    cvs_status st = set_device(c);
    if (st != CVS_OK) { delete c; return st; }
    st = ctx_alloc(c, &c->qkey, 257 * sizeof(long long));
    if (st == CVS_OK) st = ctx_alloc(c, &c->counters, kNumCounters * sizeof(unsigned long long));
    if (st == CVS_OK) st = ctx_alloc(c, &c->d_status, sizeof(int));
    if (st == CVS_OK) st = ctx_alloc(c, &c->d_rgb1, 16);
    if (st == CVS_OK) st = ctx_alloc(c, &c->d_probe, 64);
    if (st != CVS_OK) {
        const std::string msg = g_err;
        cvs_destroy(c);
        return fail(st, "cvs_create: %s", msg.c_str());
    }
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_counters, kNumCounters * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_mid);
    if (e == cudaSuccess) e = copy_qkeys_to(c->qkey, c->own);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->own);
    if (e != cudaSuccess) {
        cvs_destroy(c);
        return fail(CVS_ERR_CUDA, "cvs_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return CVS_OK;
}

void cvs_destroy(cvs_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->own) cudaStreamSynchronize(c->own);
    cudaDeviceSynchronize();
    drop_graphs(c);
    for (auto& kv : c->owned) cudaFree(kv.first);  // every buffer the context allocated
    c->owned.clear();
    c->in_use = 0;
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->h_counters) cudaFreeHost(c->h_counters);
    if (c->h_unique) cudaFreeHost(c->h_unique);
    if (c->h_arc_probe) cudaFreeHost(c->h_arc_probe);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->ev_mid) cudaEventDestroy(c->ev_mid);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

cvs_status cvs_set_option(cvs_ctx* c, const char* name, double value) {
    if (!c || !name) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (!std::strcmp(name, "fp32_window")) {
        if (!(value > 0.0 && value < 0.25))
            return fail(CVS_ERR_INVALID_ARG, "fp32_window must be in (0, 0.25)");
        c->window = value;
    } else if (!std::strcmp(name, "block")) {
        const int v = (int)value;
        if (v != 64 && v != kSearchBlock)
            return fail(CVS_ERR_INVALID_ARG, "block must be 64 or %d", kSearchBlock);
        c->shape.block = v;
    } else if (!std::strcmp(name, "blocks_per_sm")) {
        if (value < 0 || value > 32) return fail(CVS_ERR_INVALID_ARG, "blocks_per_sm in [0, 32]");
        c->shape.blocks_per_sm = (int)value;
    } else if (!std::strcmp(name, "kchunk")) {
        if (value < 0 || value > kMaxGrid) return fail(CVS_ERR_INVALID_ARG, "kchunk in [0, %d]", kMaxGrid);
        c->shape.kchunk = (int)value;
    } else if (!std::strcmp(name, "autotune")) {
        if (value != 0 && value != 1) return fail(CVS_ERR_INVALID_ARG, "autotune is 0 or 1");
        c->autotune = (int)value;
    } else if (!std::strcmp(name, "graphs")) {
        if (value != 0 && value != 1) return fail(CVS_ERR_INVALID_ARG, "graphs is 0 or 1");
        c->use_graphs = (int)value;
        if (!c->use_graphs) drop_graphs(c);
    } else if (!std::strcmp(name, "dedup")) {
        if (value != 0 && value != 1 && value != 2)
            return fail(CVS_ERR_INVALID_ARG, "dedup is 0, 1 or 2");
        if (value == 1) {  // its tables, now rather than inside a later search
            CVS_CUDA(cudaSetDevice(c->device));
            cvs_status ds = ensure_dedup(c);
            if (ds != CVS_OK) return ds;
        }
        c->dedup = (int)value;
    } else if (!std::strcmp(name, "fp64_fallback")) {
        if (value != 0 && value != 1) return fail(CVS_ERR_INVALID_ARG, "fp64_fallback is 0 or 1");
        c->fp64_fallback = (int)value;
    } else if (!std::strcmp(name, "list_batch_items")) {
        if (!(value >= 1 && value <= (double)(int64_t(1) << 26)))
            return fail(CVS_ERR_INVALID_ARG, "list_batch_items in [1, 2^26]");
        c->list_batch_items = (int64_t)value;
    } else if (!std::strcmp(name, "angle_ranges")) {
        if (value != 0 && value != 1 && value != 2)
            return fail(CVS_ERR_INVALID_ARG, "angle_ranges is 0, 1 or 2");
        c->angle_ranges = (int)value;
        const int arcs = c->grid.arcs_ok && c->angle_ranges;
        if (arcs != c->grid.arcs) {
            drop_graphs(c);
            c->grid.arcs = arcs;
            c->tuned.clear();
        }
    } else {
        return fail(CVS_ERR_INVALID_ARG, "unknown option '%s'", name);
    }
    return CVS_OK;
}

cvs_status cvs_get_option(cvs_ctx* c, const char* name, double* value) {
    if (!c || !name || !value) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (!std::strcmp(name, "fp32_window")) *value = c->window;
    else if (!std::strcmp(name, "block")) *value = c->shape.block;
    else if (!std::strcmp(name, "blocks_per_sm")) *value = c->shape.blocks_per_sm;
    else if (!std::strcmp(name, "kchunk")) *value = c->shape.kchunk;
    else if (!std::strcmp(name, "autotune")) *value = c->autotune;
    else if (!std::strcmp(name, "graphs")) *value = c->use_graphs;
    else if (!std::strcmp(name, "dedup")) *value = c->dedup;
    else if (!std::strcmp(name, "angle_ranges")) *value = c->angle_ranges;
    else if (!std::strcmp(name, "list_batch_items")) *value = (double)c->list_batch_items;
    else if (!std::strcmp(name, "fp64_fallback")) *value = c->fp64_fallback;
    else if (!std::strcmp(name, "graph_launches")) *value = (double)c->graph_launches;
    else if (!std::strcmp(name, "graphs_cached")) *value = (double)c->graphs.size();
    else if (!std::strcmp(name, "mem_in_use")) *value = (double)c->in_use;
    else if (!std::strcmp(name, "mem_budget")) *value = (double)c->budget;
    else return fail(CVS_ERR_INVALID_ARG, "unknown option '%s'", name);
    return CVS_OK;
}

cvs_status cvs_signal_bounds(const cvs_thresholds* thr, int32_t* hi_min, int32_t* lo_max) {
    cvs_status st = check_thresholds(thr);
    if (st != CVS_OK) return st;
    if (!hi_min || !lo_max) return fail(CVS_ERR_INVALID_ARG, "output pointer is NULL");
    thresholds_to_int(thr, hi_min, lo_max);
    return CVS_OK;
}

cvs_status cvs_trig_table(cvs_ctx* c, const double* angles, int32_t n, double* s, double* co) {
    if (!c || !angles || !s || !co) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0 || n > kMaxGrid) return fail(CVS_ERR_INVALID_ARG, "n must be in [1, %d]", kMaxGrid);
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(angles[i])) return fail(CVS_ERR_INVALID_ARG, "angle %d not finite", i);
    cvs_status st0 = set_device(c);
    if (st0 != CVS_OK) return st0;
    double *da = nullptr, *ds = nullptr, *dc = nullptr;
    float2* dsc = nullptr;
    cudaStream_t st = c->own;
    CVS_TRY(ctx_alloc(c, &da, sizeof(double) * n * 3 + sizeof(float2) * n));
    ds = da + n;
    dc = ds + n;
    dsc = reinterpret_cast<float2*>(dc + n);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(da, angles, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_trig_table(da, n, ds, dc, dsc, c->d_status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s, ds, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(co, dc, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ctx_free(c, da);
    if (e != cudaSuccess) return fail(CVS_ERR_CUDA, "cvs_trig_table: %s", cudaGetErrorString(e));
    if (status) return fail(CVS_ERR_NUMERIC, "an angle's sine could not be certified");
    return CVS_OK;
}

cvs_status cvs_target_lab(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n, double* lab_dev,
                          void* stream) {
    if (!c || (n > 0 && (!rgb_dev || !lab_dev))) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(CVS_ERR_INVALID_ARG, "n must be >= 0");
    cvs_status st0 = set_device(c);
    if (st0 != CVS_OK) return st0;
    CVS_CUDA(launch_target_lab(rgb_dev, n, lab_dev, (cudaStream_t)stream));
    return CVS_OK;
}

}  // extern "C"

namespace {

// Every passing pair of n colours on the device (grid and thresholds
// prepared by the caller), per batch of colours: the search leaves each work
// item's passing-slot bitmap and count; a scan of the counts gives each
// item's first record; the emit kernel writes the records, in (target, k, m)
// order, straight to out (records at or beyond cap are not written).  Fills
// offs_host (n + 1 entries).  Synchronous on st.
cvs_status search_pairs(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n, const cvs_thresholds* thr,
                        cvs_precision prec, cvs_pair* out, int64_t cap, uint32_t target0,
                        int64_t* offs_host, cudaStream_t st) {
    const int K = c->grid.K, H = c->grid.H;
    // radii per work item: the automatic choice, at least 1024 slots (an item
    // has a fixed cost in the search and in the emit kernel), and within the
    // bitmap of a warp
    int kchunk = choose_kchunk(c, n, K, H);
    if (c->shape.kchunk == 0 && kchunk * H < 1024) kchunk = (1024 + H - 1) / H;
    if (kchunk > K) kchunk = K;
    const int kmax = kListMaxSlots / H > 0 ? kListMaxSlots / H : 1;
    if (kchunk > kmax) kchunk = kmax;
    if (kchunk > kListMaxRadii) kchunk = kListMaxRadii;
    const int64_t n_kc = (K + kchunk - 1) / kchunk;
    const int words = (kchunk * H + 31) / 32;
    // targets per batch: within list_batch_items work items and 256 MiB of bitmaps
    int64_t items = c->list_batch_items;
    const int64_t by_bytes = ((int64_t)256 << 20) / (4 * (int64_t)words);
    if (items > by_bytes) items = by_bytes;
    int64_t nb = items / n_kc;
    nb = nb < 1 ? 1 : (nb > n ? n : nb);
    const int64_t nitems = nb * n_kc;
    CVS_TRY(ensure_targets(c, nb));
    CVS_TRY(grow(c, &c->d_offs, &c->cap_offs, n + 1));
    CVS_TRY(grow(c, &c->d_bits, &c->cap_bits, nitems * words));
    CVS_TRY(grow(c, &c->d_icount, &c->cap_icount, nitems));
    CVS_TRY(grow(c, &c->d_within, &c->cap_within, nitems));
    CVS_TRY(grow(c, &c->d_tiles, &c->cap_tiles, (nitems + 4095) / 4096));
    CVS_CUDA(cudaMemsetAsync(c->d_offs, 0, sizeof(int64_t), st));
    ListOut lo;
    lo.item_bits = c->d_bits;
    lo.item_words = words;
    lo.item_count = c->d_icount;
    lo.kchunk = kchunk;
    EmitArgs e{};
    e.tf = c->tf;
    e.td = c->td;
    e.grid = c->grid;
    e.qkey = c->qkey;
    thresholds_to_int(thr, &e.hi_min, &e.lo_max);
    e.mask2 = thr->pattern_mask << 1;
    e.clip = thr->gamut_mode;
    e.half_w = (float)(0.5 - c->window);
    e.prec = (int32_t)prec;
    e.kchunk = kchunk;
    e.item_bits = c->d_bits;
    e.item_words = words;
    e.item_base = c->d_within;
    e.tile_base = c->d_tiles;
    e.out = out;
    e.out_cap = cap;
    for (int64_t t0 = 0; t0 < n; t0 += nb) {
        const int64_t b = n - t0 < nb ? n - t0 : nb;
        CVS_CUDA(launch_setup_colors(rgb_dev + 3 * t0, b, c->grid.rmax, c->tf, c->td, c->acc, st));
        c->search_kind = 0;
        CVS_TRY(run_search(c, b, thr, prec, 1, target0 + (uint32_t)t0, st, false, &lo));
        CVS_CUDA(launch_pair_scan(c->d_icount, c->grid.sym, b * n_kc, c->d_within, c->d_tiles,
                                  c->d_offs + t0, st));
        e.n_targets = b;
        e.offs = c->d_offs + t0;
        e.target_id = target0 + (uint32_t)t0;
        CVS_CUDA(launch_emit_pairs(e, c->num_sms, st));
    }
    CVS_CUDA(cudaMemcpyAsync(offs_host, c->d_offs, sizeof(int64_t) * (size_t)(n + 1),
                             cudaMemcpyDeviceToHost, st));
    CVS_CUDA(cudaStreamSynchronize(st));
    collect_stats(c);
    return CVS_OK;
}

}  // namespace

extern "C" {

cvs_status cvs_search_color(cvs_ctx* c, const uint8_t rgb[3], uint32_t target,
                            const cvs_grid* grid, const cvs_thresholds* thr, cvs_precision prec,
                            cvs_pair* out_host, size_t cap, size_t* n_out) {
    if (!c || !rgb || !n_out || (cap > 0 && !out_host))
        return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    if (st0 != CVS_OK) return st0;
    const int64_t nd = (int64_t)c->grid.K * c->grid.N;  // most pairs one colour can have
    CVS_TRY(grow(c, &c->compact, &c->cap_compact, nd));
    cudaStream_t st = c->own;
    CVS_CUDA(cudaMemcpyAsync(c->d_rgb1, rgb, 3, cudaMemcpyHostToDevice, st));
    int64_t offs[2] = {0, 0};
    st0 = search_pairs(c, c->d_rgb1, 1, thr, prec, c->compact, nd, target, offs, st);
    if (st0 != CVS_OK) return st0;
    const int64_t n = offs[1];
    *n_out = (size_t)n;
    const size_t ncopy = (size_t)n < cap ? (size_t)n : cap;
    if (ncopy)
        CVS_CUDA(cudaMemcpy(out_host, c->compact, ncopy * sizeof(cvs_pair), cudaMemcpyDeviceToHost));
    if ((size_t)n > cap)
        return fail(CVS_ERR_TRUNCATED, "%lld passing pairs, capacity %zu", (long long)n, cap);
    return CVS_OK;
}

cvs_status cvs_search_colors_pairs(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n,
                                   const cvs_grid* grid, const cvs_thresholds* thr,
                                   cvs_precision prec, cvs_pair* out_dev, int64_t cap,
                                   int64_t* offsets_host, int64_t* n_out, void* stream) {
    if (!c || !n_out || (cap > 0 && !out_dev)) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    *n_out = 0;
    if (n < 0 || n > ((int64_t)1 << 31)) return fail(CVS_ERR_INVALID_ARG, "n out of range");
    if (cap < 0) return fail(CVS_ERR_INVALID_ARG, "negative capacity");
    if (n > 0 && !rgb_dev) return fail(CVS_ERR_INVALID_ARG, "NULL device buffer");
    if (cap > 0 && (reinterpret_cast<uintptr_t>(out_dev) & 15u))
        return fail(CVS_ERR_INVALID_ARG, "out_dev must be 16-byte aligned");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    if (st0 != CVS_OK) return st0;
    if (offsets_host) offsets_host[0] = 0;
    if (n == 0) return CVS_OK;
    std::vector<int64_t> offs((size_t)n + 1);
    st0 = search_pairs(c, rgb_dev, n, thr, prec, out_dev, cap, 0, offs.data(),
                       (cudaStream_t)stream);
    if (st0 != CVS_OK) return st0;
    if (offsets_host) std::memcpy(offsets_host, offs.data(), sizeof(int64_t) * ((size_t)n + 1));
    const int64_t total = offs[n];
    *n_out = total;
    if (total > cap)
        return fail(CVS_ERR_TRUNCATED, "%lld passing pairs, capacity %lld", (long long)total,
                    (long long)cap);
    return CVS_OK;
}

cvs_status cvs_search_colors(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n, const cvs_grid* grid,
                             const cvs_thresholds* thr, cvs_precision prec,
                             const cvs_capacity_map* out, void* stream) {
    if (!c || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > (int64_t)1 << 40) return fail(CVS_ERR_INVALID_ARG, "n out of range");
    if (n > 0 && (!rgb_dev || !out->max_r || !out->count || !out->pmask))
        return fail(CVS_ERR_INVALID_ARG, "NULL device buffer");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    if (st0 == CVS_OK) st0 = ensure_targets(c, n);
    if (st0 != CVS_OK) return st0;
    if (n == 0) return CVS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    auto enqueue = [&](cudaStream_t s, ImageDesc*) -> cvs_status {
        CVS_CUDA(launch_setup_colors(rgb_dev, n, c->grid.rmax, c->tf, c->td, c->acc, s));
        c->search_kind = 0;
        cvs_status r = run_search(c, n, thr, prec, 0, 0, s, s == c->cap);
        if (r != CVS_OK) return r;
        CVS_CUDA(launch_finalize_colors(c->acc, n, out->max_r, out->count, out->pmask, s));
        return CVS_OK;
    };
    if (!c->use_graphs) return enqueue(st, nullptr);
    if (c->autotune) {  // tune outside the capture, once
        const auto key = tune_key(c, n, (int)prec, thr->gamut_mode, 0);
        if (!c->tuned.count(key)) {
            st0 = enqueue(st, nullptr);
            if (st0 != CVS_OK) return st0;
        }
    }
    std::vector<uint64_t> key = {1, (uint64_t)rgb_dev, (uint64_t)n, (uint64_t)out->max_r,
                                 (uint64_t)out->count, (uint64_t)out->pmask, dbits(thr->v_th),
                                 dbits(thr->r_novib), thr->pattern_mask,
                                 (uint64_t)thr->gamut_mode, (uint64_t)prec,
                                 (uint64_t)c->shape.block, (uint64_t)c->shape.blocks_per_sm,
                                 (uint64_t)c->shape.kchunk, dbits(c->window),
                                 dbits(thr->max_dl)};
    st0 = graph_launch(c, key, st, enqueue);
    if (st0 == CVS_OK) c->last_pending = true;
    return st0;
}

cvs_status cvs_search_colors_multi(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n,
                                   const cvs_grid* grid, const cvs_thresholds* thr,
                                   int32_t n_thr, cvs_precision prec,
                                   const cvs_capacity_map* out, void* stream) {
    if (!c || !out || !thr) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > (int64_t)1 << 36) return fail(CVS_ERR_INVALID_ARG, "n out of range");
    if (n_thr < 1 || n_thr > kMaxThresholdSets)
        return fail(CVS_ERR_INVALID_ARG, "n_thr = %d, must be in [1, %d]", (int)n_thr,
                    kMaxThresholdSets);
    if (n > 0 && (!rgb_dev || !out->max_r || !out->count || !out->pmask))
        return fail(CVS_ERR_INVALID_ARG, "NULL device buffer");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    for (int s = 0; s < n_thr && st0 == CVS_OK; ++s) {
        st0 = check_thresholds(thr + s);
        if (st0 == CVS_OK && thr[s].gamut_mode != thr[0].gamut_mode)
            st0 = fail(CVS_ERR_INVALID_ARG, "threshold set %d: gamut_mode differs from set 0", s);
    }
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    for (int s = 0; s < n_thr && st0 == CVS_OK; ++s) st0 = ensure_ltab(c, thr + s);
    if (st0 == CVS_OK) st0 = ensure_targets(c, n);
    if (st0 != CVS_OK) return st0;
    if (n == 0) return CVS_OK;
    CVS_TRY(grow(c, &c->acc_multi, &c->cap_acc_multi, n * n_thr));
    MultiArgs a{};
    a.tf = c->tf;
    a.td = c->td;
    a.order = c->d_order;
    a.acc = c->acc_multi;
    a.n_targets = n;
    a.grid = c->grid;
    a.qkey = c->qkey;
    a.n_thr = n_thr;
    a.hi_min_all = 256;
    a.all_patterns = 1;
    for (int s = 0; s < n_thr; ++s) {
        thresholds_to_int(thr + s, &a.hi_min[s], &a.lo_max[s]);
        for (int p = 1; p <= 7; ++p)
            if ((thr[s].pattern_mask >> (p - 1)) & 1u) a.pmask_sets[p] |= 1u << s;
        if ((thr[s].pattern_mask & 0x7Fu) != 0x7Fu) a.all_patterns = 0;
        a.hi_min_all = a.hi_min[s] < a.hi_min_all ? a.hi_min[s] : a.hi_min_all;
    }
    a.clip = thr[0].gamut_mode;
    // luminance limits: per set, sets without one pass it always
    a.ltab = nullptr;
    a.dl_free = 0;
    for (int s = 0; s < n_thr; ++s) {
        if (dl_on(thr + s)) {
            a.ltab = c->ltab;
            std::memcpy(&a.max_dl_bits[s], &thr[s].max_dl, sizeof(double));
        } else {
            a.dl_free |= 1u << s;
            a.max_dl_bits[s] = -1;  // never consulted: the set is in dl_free
        }
    }
    a.half_w = (float)(0.5 - c->window);
    a.prec = (int32_t)prec;
    a.kchunk = choose_kchunk(c, n, c->grid.K, c->grid.H);
    if (a.kchunk > multi_max_chunk()) a.kchunk = multi_max_chunk();
    a.work_counter = c->counters;
    a.stats = c->counters + 1;
    a.num_sms = c->num_sms;
    cudaStream_t st = (cudaStream_t)stream;
    CVS_CUDA(launch_setup_colors(rgb_dev, n, c->grid.rmax, c->tf, c->td, c->acc, st));
    // angle ranges of the union of the sets (the smallest hi_min, every
    // enabled pattern): a superset of the slots that pass any set
    a.arc_ranges = nullptr;
    a.arc_cap = 0;
    a.ev_ranges = nullptr;
    if (prec == CVS_PREC_FP32_RECHECK && !a.clip && c->grid.arcs) {
        SearchArgs pa{};
        pa.tf = c->tf;
        pa.td = c->td;
        pa.grid = c->grid;
        pa.hi_min = a.hi_min_all;
        pa.lo_max = -1;
        for (int p = 1; p <= 7; ++p)
            if (a.pmask_sets[p]) pa.mask2 |= 1u << p;
        pa.num_sms = c->num_sms;
        c->search_kind = 0;
        CVS_TRY(prepare_arcs(c, pa, n, prec, kMultiArcKey, st, false));
        if (pa.grid.arcs && pa.arc_ranges && pa.arc_cap >= c->grid.K) {
            a.arc_ranges = pa.arc_ranges;
            a.arc_cap = pa.arc_cap;
            a.ev_ranges = c->ev_mid;
            a.ev_flags = cudaEventRecordDefault;
        }
    }
    CVS_CUDA(launch_init_acc(c->acc_multi, n * n_thr, st));
    CVS_CUDA(cudaMemsetAsync(c->counters, 0, kNumCounters * sizeof(unsigned long long), st));
    c->last_arcs = a.arc_ranges != nullptr;
    CVS_CUDA(cudaEventRecord(c->ev0, st));
    CVS_CUDA(launch_search_multi(a, st));
    CVS_CUDA(cudaEventRecord(c->ev1, st));
    CVS_CUDA(cudaMemcpyAsync(c->h_counters, c->counters, kNumCounters * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, st));
    CVS_CUDA(launch_finalize_colors(c->acc_multi, n * n_thr, out->max_r, out->count, out->pmask,
                                    st));
    cvs_stats& s = c->last;
    s = cvs_stats{};
    s.targets = n;
    s.candidates = n * (int64_t)c->grid.K * c->grid.N;
    s.colors_fp32 = prec == CVS_PREC_FP64 ? 0 : s.candidates;
    s.symmetric = c->grid.sym;
    s.precision = (int32_t)prec;
    c->last_pending = true;
    return CVS_OK;
}

cvs_status cvs_search_colors_host(cvs_ctx* c, const uint8_t* rgb_host, int64_t n,
                                  const cvs_grid* grid, const cvs_thresholds* thr,
                                  cvs_precision prec, float* max_r_host, int32_t* count_host,
                                  uint8_t* pmask_host) {
    if (!c) return fail(CVS_ERR_INVALID_ARG, "NULL context");
    if (n < 0) return fail(CVS_ERR_INVALID_ARG, "n must be >= 0");
    if (n > 0 && (!rgb_host || !max_r_host || !count_host || !pmask_host))
        return fail(CVS_ERR_INVALID_ARG, "NULL host buffer");
    cvs_status st0 = set_device(c);
    if (st0 != CVS_OK) return st0;
    CVS_TRY(grow(c, &c->d_in, &c->cap_in, 3 * n));
    CVS_TRY(grow(c, &c->d_maxr, &c->cap_maxr, n));
    CVS_TRY(grow(c, &c->d_count, &c->cap_count, n));
    CVS_TRY(grow(c, &c->d_pmask, &c->cap_pmask, n));
    cudaStream_t st = c->own;
    if (n > 0) CVS_CUDA(cudaMemcpyAsync(c->d_in, rgb_host, 3 * n, cudaMemcpyHostToDevice, st));
    cvs_capacity_map m{c->d_maxr, c->d_count, c->d_pmask};
    st0 = cvs_search_colors(c, c->d_in, n, grid, thr, prec, &m, st);
    if (st0 != CVS_OK) return st0;
    if (n > 0) {
        CVS_CUDA(cudaMemcpyAsync(max_r_host, c->d_maxr, 4 * n, cudaMemcpyDeviceToHost, st));
        CVS_CUDA(cudaMemcpyAsync(count_host, c->d_count, 4 * n, cudaMemcpyDeviceToHost, st));
        CVS_CUDA(cudaMemcpyAsync(pmask_host, c->d_pmask, n, cudaMemcpyDeviceToHost, st));
    }
    CVS_CUDA(cudaStreamSynchronize(st));
    collect_stats(c);
    return CVS_OK;
}

cvs_status cvs_search_images(cvs_ctx* c, const cvs_image* batch, int32_t n, const cvs_grid* grid,
                             const cvs_thresholds* thr, cvs_precision prec,
                             const cvs_capacity_map* maps, void* stream) {
    if (!c || !batch || !maps) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0 || n > (1 << 20)) return fail(CVS_ERR_INVALID_ARG, "n must be in [1, 2^20]");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    std::vector<ImageDesc> h(n);
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const cvs_image& im = batch[i];
        if (!im.rgb || im.width <= 0 || im.height <= 0 || im.pitch_bytes < 3LL * im.width)
            return fail(CVS_ERR_INVALID_ARG, "image %d: bad pointer, size or pitch", i);
        if (!maps[i].max_r || !maps[i].count || !maps[i].pmask)
            return fail(CVS_ERR_INVALID_ARG, "map %d: NULL buffer", i);
        const int64_t px = (int64_t)im.width * im.height;
        if (px >= ((int64_t)1 << 40)) return fail(CVS_ERR_INVALID_ARG, "image %d too large", i);
        h[i] = ImageDesc{im.rgb, im.pitch_bytes, im.width, im.height, total,
                         maps[i].max_r, maps[i].count, maps[i].pmask};
        total += px;
    }
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    if (st0 != CVS_OK) return st0;
    const bool auto_dedup =
        c->dedup == 2 && !c->use_graphs && total >= kDedupAutoPixels;
    // One search per distinct colour of the batch.  Every allocation comes
    // before the gather, the only write to the maps.
    auto search_distinct = [&]() -> cvs_status {
        CVS_TRY(ensure_dedup(c));
        cudaStream_t st = (cudaStream_t)stream;
        CVS_TRY(grow(c, &c->d_imgs, &c->cap_imgs, n));
        CVS_CUDA(cudaMemcpyAsync(c->d_imgs, h.data(), sizeof(ImageDesc) * n,
                                 cudaMemcpyHostToDevice, st));
        CVS_CUDA(launch_dedup_mark(c->d_imgs, n, total, c->d_present, st));
        CVS_CUDA(launch_dedup_scan(c->d_present, c->d_scan, c->d_scan + 1024, c->d_index,
                                   c->d_unique, st));
        CVS_CUDA(cudaMemcpyAsync(c->h_unique, c->d_scan + 1024, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
        CVS_CUDA(cudaStreamSynchronize(st));
        const int64_t nu = *c->h_unique;
        CVS_TRY(ensure_targets(c, nu));  // the search covers the distinct colours only
        CVS_CUDA(launch_setup_colors(c->d_unique, nu, c->grid.rmax, c->tf, c->td, c->acc, st));
        c->search_kind = 1;
        st0 = run_search(c, nu, thr, prec, 0, 0, st);
        if (st0 != CVS_OK) return st0;
        CVS_CUDA(launch_dedup_gather(c->d_imgs, n, total, c->d_index, c->acc, st));
        return CVS_OK;
    };
    if (c->dedup == 1) return search_distinct();
    if (auto_dedup) {
        st0 = search_distinct();
        if (st0 != CVS_ERR_NO_MEMORY) return st0;
        drop_dedup(c);  // memory the budget refused: the per-pixel search, tables freed
        g_err.clear();
    }
    st0 = ensure_targets(c, total);
    if (st0 != CVS_OK) return st0;
    cudaStream_t st = (cudaStream_t)stream;
    auto enqueue = [&](cudaStream_t s, ImageDesc* d_imgs) -> cvs_status {
        CVS_CUDA(launch_setup_images(d_imgs, n, total, c->grid.rmax, c->tf, c->td, c->acc, s));
        c->search_kind = 1;
        cvs_status r = run_search(c, total, thr, prec, 0, 0, s, s == c->cap);
        if (r != CVS_OK) return r;
        CVS_CUDA(launch_finalize_images(c->acc, c->td, total, d_imgs, s));
        return CVS_OK;
    };
    if (!c->use_graphs) {
        CVS_TRY(grow(c, &c->d_imgs, &c->cap_imgs, n));
        CVS_CUDA(cudaMemcpyAsync(c->d_imgs, h.data(), sizeof(ImageDesc) * n, cudaMemcpyHostToDevice,
                                 st));
        return enqueue(st, c->d_imgs);
    }
    std::vector<uint64_t> key = {2, (uint64_t)n, dbits(thr->v_th), dbits(thr->r_novib),
                                 thr->pattern_mask, (uint64_t)thr->gamut_mode, (uint64_t)prec,
                                 (uint64_t)c->shape.block, (uint64_t)c->shape.blocks_per_sm,
                                 (uint64_t)c->shape.kchunk, dbits(c->window),
                                 dbits(thr->max_dl)};
    for (const ImageDesc& d : h) {
        key.insert(key.end(), {(uint64_t)d.rgb, (uint64_t)d.pitch, (uint64_t)d.width,
                               (uint64_t)d.height, (uint64_t)d.max_r, (uint64_t)d.count,
                               (uint64_t)d.pmask});
    }
    st0 = graph_launch(c, key, st, enqueue, &h);
    if (st0 == CVS_OK) c->last_pending = true;
    return st0;
}

cvs_status cvs_embed_image(cvs_ctx* c, const cvs_image* img, const uint8_t* pattern_dev,
                           int64_t pattern_pitch, const cvs_grid* grid, const cvs_thresholds* thr,
                           cvs_precision prec, uint8_t* frame_a_dev, uint8_t* frame_b_dev,
                           int64_t frame_pitch, uint32_t* choice_dev, void* stream) {
    if (!c || !img || !pattern_dev || !frame_a_dev || !frame_b_dev)
        return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (!img->rgb || img->width <= 0 || img->height <= 0 || img->pitch_bytes < 3LL * img->width)
        return fail(CVS_ERR_INVALID_ARG, "bad image pointer, size or pitch");
    if (pattern_pitch < img->width) return fail(CVS_ERR_INVALID_ARG, "pattern pitch < width");
    if (frame_pitch < 3LL * img->width) return fail(CVS_ERR_INVALID_ARG, "frame pitch < 3 * width");
    if (frame_a_dev == frame_b_dev) return fail(CVS_ERR_INVALID_ARG, "the two frames must differ");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    const int64_t px = (int64_t)img->width * img->height;
    if (px >= ((int64_t)1 << 40)) return fail(CVS_ERR_INVALID_ARG, "image too large");
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    if (st0 == CVS_OK) st0 = ensure_targets(c, px);
    if (st0 != CVS_OK) return st0;
    cudaStream_t st = (cudaStream_t)stream;
    const ImageDesc h{img->rgb, img->pitch_bytes, img->width, img->height, 0, nullptr, nullptr,
                      nullptr};
    CVS_TRY(grow(c, &c->d_imgs, &c->cap_imgs, 1));
    CVS_CUDA(cudaMemcpyAsync(c->d_imgs, &h, sizeof(ImageDesc), cudaMemcpyHostToDevice, st));
    CVS_CUDA(launch_setup_images(c->d_imgs, 1, px, c->grid.rmax, c->tf, c->td, c->acc, st));
    EmbedArgs a{};
    a.tf = c->tf;
    a.td = c->td;
    a.n = px;
    a.rgb = img->rgb;
    a.pitch = img->pitch_bytes;
    a.width = img->width;
    a.height = img->height;
    a.pattern = pattern_dev;
    a.pattern_pitch = pattern_pitch;
    a.frame_a = frame_a_dev;
    a.frame_b = frame_b_dev;
    a.frame_pitch = frame_pitch;
    a.choice = choice_dev;
    a.grid = c->grid;
    a.order = c->d_order;
    a.qkey = c->qkey;
    thresholds_to_int(thr, &a.hi_min, &a.lo_max);
    a.mask2 = thr->pattern_mask << 1;
    a.clip = thr->gamut_mode;
    a.ltab = dl_on(thr) ? c->ltab : nullptr;
    a.max_dl = thr->max_dl;
    a.half_w = (float)(0.5 - c->window);
    a.prec = (int32_t)prec;
    a.work_counter = c->counters;
    a.stats = c->counters + 1;
    a.num_sms = c->num_sms;
    CVS_CUDA(cudaMemsetAsync(c->counters, 0, kNumCounters * sizeof(unsigned long long), st));
    c->last_arcs = false;
    CVS_CUDA(cudaEventRecord(c->ev0, st));
    CVS_CUDA(launch_embed(a, st));
    CVS_CUDA(cudaEventRecord(c->ev1, st));
    CVS_CUDA(cudaMemcpyAsync(c->h_counters, c->counters, kNumCounters * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, st));
    cvs_stats& s = c->last;
    s = cvs_stats{};
    s.targets = px;
    s.symmetric = c->grid.sym;
    s.precision = (int32_t)prec;
    c->last_pending = true;
    return CVS_OK;
}

cvs_status cvs_autotune(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n, const cvs_grid* grid,
                        const cvs_thresholds* thr, cvs_precision prec, cvs_launch_shape* best) {
    if (!c || !rgb_dev || !best) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0) return fail(CVS_ERR_INVALID_ARG, "n must be > 0");
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    if (st0 == CVS_OK) st0 = ensure_targets(c, n);
    if (st0 != CVS_OK) return st0;
    cudaStream_t st = c->own;
    CVS_CUDA(launch_setup_colors(rgb_dev, n, c->grid.rmax, c->tf, c->td, c->acc, st));
    SearchArgs a{};
    a.tf = c->tf;
    a.td = c->td;
    a.acc = c->acc;
    a.n_targets = n;
    a.grid = c->grid;
    a.qkey = c->qkey;
    thresholds_to_int(thr, &a.hi_min, &a.lo_max);
    a.mask2 = thr->pattern_mask << 1;
    a.clip = thr->gamut_mode;
    a.half_w = (float)(0.5 - c->window);
    a.prec = (int32_t)prec;
    a.num_sms = c->num_sms;
    c->search_kind = 0;
    st0 = prepare_arcs(c, a, n, prec, 0, st, false);  // tune the walk the search will take
    if (st0 != CVS_OK) return st0;
    LaunchShape sh;
    double ms = 0.0;
    st0 = tune_shape(c, a, st, &sh, &ms);
    if (st0 != CVS_OK) return st0;
    c->tuned[tune_key(c, n, (int)prec, a.clip, 0)] = sh;
    best->block = sh.block;
    best->blocks_per_sm = sh.blocks_per_sm;
    best->kchunk = sh.kchunk;
    best->reserved = 0;
    best->ms = ms;
    return CVS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ capacity table
struct cvs_lut {
    int device = 0;
    uint64_t* entry = nullptr;   // 2^24: (count << 32) | max_r bits
    uint8_t* pmask = nullptr;    // 2^24
};

extern "C" {

cvs_status cvs_lut_build(cvs_ctx* c, const cvs_grid* grid, const cvs_thresholds* thr,
                         cvs_precision prec, cvs_lut** out, void* stream) {
    if (!c || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    constexpr int64_t kColours = int64_t(1) << 24, kChunk = int64_t(1) << 22;
    if (st0 == CVS_OK) st0 = ensure_targets(c, kChunk);
    if (st0 != CVS_OK) return st0;
    cvs_lut* L = new cvs_lut();
    L->device = c->device;
    uint8_t* rgb = nullptr;
    // the table belongs to the caller; the colour buffer is the context's scratch
    cudaError_t e = cudaMalloc(&L->entry, sizeof(uint64_t) * kColours);
    if (e == cudaSuccess) e = cudaMalloc(&L->pmask, kColours);
    if (e != cudaSuccess) {
        cvs_lut_destroy(L);
        return fail(e == cudaErrorMemoryAllocation ? CVS_ERR_NO_MEMORY : CVS_ERR_CUDA,
                    "cvs_lut_build: %s", cudaGetErrorString(e));
    }
    st0 = ctx_alloc(c, &rgb, 3 * kChunk);
    if (st0 != CVS_OK) {
        cvs_lut_destroy(L);
        return st0;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t first = 0; first < kColours && st0 == CVS_OK; first += kChunk) {
        e = launch_rgb_iota(rgb, first, kChunk, st);
        if (e == cudaSuccess) e = launch_setup_colors(rgb, kChunk, c->grid.rmax, c->tf, c->td, c->acc, st);
        if (e != cudaSuccess) { st0 = fail(CVS_ERR_CUDA, "cvs_lut_build: %s", cudaGetErrorString(e)); break; }
        c->search_kind = 2;
        st0 = run_search(c, kChunk, thr, prec, 0, 0, st);
        if (st0 != CVS_OK) break;
        e = launch_lut_pack(c->acc, kChunk, L->entry + first, L->pmask + first, st);
        if (e != cudaSuccess) st0 = fail(CVS_ERR_CUDA, "cvs_lut_build: %s", cudaGetErrorString(e));
    }
    // the colour buffer is released once the stream has consumed it
    cudaError_t se = cudaStreamSynchronize(st);
    ctx_free(c, rgb);
    if (st0 == CVS_OK && se != cudaSuccess)
        st0 = fail(CVS_ERR_CUDA, "cvs_lut_build: %s", cudaGetErrorString(se));
    if (st0 != CVS_OK) {
        cvs_lut_destroy(L);
        return st0;
    }
    collect_stats(c);
    c->last.candidates = kColours * (int64_t)c->grid.K * c->grid.N;
    c->last.targets = kColours;
    *out = L;
    return CVS_OK;
}

void cvs_lut_destroy(cvs_lut* L) {
    if (!L) return;
    cudaSetDevice(L->device);
    cudaDeviceSynchronize();
    void* ptrs[] = {L->entry, L->pmask};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete L;
}

cvs_status cvs_lut_lookup_colors(cvs_lut* L, const uint8_t* rgb_dev, int64_t n,
                                 const cvs_capacity_map* out, void* stream) {
    if (!L || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(CVS_ERR_INVALID_ARG, "n must be >= 0");
    if (n > 0 && (!rgb_dev || !out->max_r || !out->count || !out->pmask))
        return fail(CVS_ERR_INVALID_ARG, "NULL device buffer");
    CVS_CUDA(cudaSetDevice(L->device));
    CVS_CUDA(launch_lut_gather_colors(rgb_dev, n, L->entry, L->pmask, out->max_r, out->count,
                                      out->pmask, (cudaStream_t)stream));
    return CVS_OK;
}

cvs_status cvs_lut_lookup_images(cvs_lut* L, const cvs_image* batch, int32_t n,
                                 const cvs_capacity_map* maps, void* stream) {
    if (!L || !batch || !maps) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0 || n > (1 << 20)) return fail(CVS_ERR_INVALID_ARG, "n must be in [1, 2^20]");
    for (int i = 0; i < n; ++i) {
        const cvs_image& im = batch[i];
        if (!im.rgb || im.width <= 0 || im.height <= 0 || im.pitch_bytes < 3LL * im.width)
            return fail(CVS_ERR_INVALID_ARG, "image %d: bad pointer, size or pitch", i);
        if (!maps[i].max_r || !maps[i].count || !maps[i].pmask)
            return fail(CVS_ERR_INVALID_ARG, "map %d: NULL buffer", i);
        if ((int64_t)im.width * im.height > ((int64_t)1 << 36))
            return fail(CVS_ERR_INVALID_ARG, "image %d too large", i);
    }
    CVS_CUDA(cudaSetDevice(L->device));
    cudaStream_t st = (cudaStream_t)stream;
    // descriptors travel by value, kGatherMaxImages images per launch
    for (int first = 0; first < n; first += kGatherMaxImages) {
        GatherBatch b{};
        b.n = n - first < kGatherMaxImages ? n - first : kGatherMaxImages;
        int64_t blocks = 0;
        for (int j = 0; j < b.n; ++j) {
            const cvs_image& im = batch[first + j];
            const cvs_capacity_map& m = maps[first + j];
            const int64_t px = (int64_t)im.width * im.height;
            b.img[j] = ImageDesc{im.rgb, im.pitch_bytes, im.width, im.height, 0, m.max_r, m.count,
                                 m.pmask};
            b.block_first[j] = blocks;
            blocks += (px + kGatherBlock - 1) / kGatherBlock;
        }
        if (blocks > 0x7FFFFFFFLL) return fail(CVS_ERR_INVALID_ARG, "batch too large for one launch");
        CVS_CUDA(launch_lut_gather_images(b, blocks, L->entry, L->pmask, st));
    }
    return CVS_OK;
}

}  // extern "C"

struct cvs_etab {
    int device = 0;
    uint4* entry = nullptr;  // 2^24 x 7 entries of 16 bytes (codes and choice)
};

extern "C" {

cvs_status cvs_etab_build(cvs_ctx* c, const cvs_grid* grid, const cvs_thresholds* thr,
                          cvs_precision prec, cvs_etab** out, void* stream) {
    if (!c || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = check_thresholds(thr);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = resolve_precision(c, &prec);
    if (st0 == CVS_OK && thr) st0 = ensure_ltab(c, thr);
    constexpr int64_t kColours = int64_t(1) << 24, kChunk = int64_t(1) << 22;
    if (st0 == CVS_OK) st0 = ensure_targets(c, kChunk);
    if (st0 != CVS_OK) return st0;
    cvs_etab* E = new cvs_etab();
    E->device = c->device;
    uint8_t* rgb = nullptr;
    uint32_t* keys = nullptr;  // one chunk's first-hit keys
    // the table belongs to the caller; keys and colours are the context's scratch
    cudaError_t e = cudaMalloc(&E->entry, sizeof(uint4) * 7 * kColours);
    if (e != cudaSuccess) {
        cvs_etab_destroy(E);
        return fail(e == cudaErrorMemoryAllocation ? CVS_ERR_NO_MEMORY : CVS_ERR_CUDA,
                    "cvs_etab_build: %s", cudaGetErrorString(e));
    }
    st0 = ctx_alloc(c, &keys, sizeof(uint32_t) * 7 * kChunk);
    if (st0 == CVS_OK) st0 = ctx_alloc(c, &rgb, 3 * kChunk);
    if (st0 != CVS_OK) {
        ctx_free(c, keys);
        cvs_etab_destroy(E);
        return st0;
    }
    FirstHitArgs a{};
    a.tf = c->tf;
    a.td = c->td;
    a.n_targets = kChunk;
    a.grid = c->grid;
    a.order = c->d_order;
    a.qkey = c->qkey;
    thresholds_to_int(thr, &a.hi_min, &a.lo_max);
    a.mask2 = thr->pattern_mask << 1;
    a.clip = thr->gamut_mode;
    a.ltab = dl_on(thr) ? c->ltab : nullptr;
    a.max_dl = thr->max_dl;
    a.half_w = (float)(0.5 - c->window);
    a.prec = (int32_t)prec;
    a.kchunk = choose_kchunk(c, kChunk, c->grid.K, c->grid.H);
    a.work_counter = c->counters;
    a.stats = c->counters + 1;
    a.num_sms = c->num_sms;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(c->counters, 0, kNumCounters * sizeof(unsigned long long), st);
    c->last_arcs = false;
    if (e == cudaSuccess) e = cudaEventRecord(c->ev0, st);
    for (int64_t first = 0; first < kColours && e == cudaSuccess; first += kChunk) {
        a.key = keys;
        e = launch_rgb_iota(rgb, first, kChunk, st);
        if (e == cudaSuccess)
            e = launch_setup_colors(rgb, kChunk, c->grid.rmax, c->tf, c->td, c->acc, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(a.key, 0xFF, sizeof(uint32_t) * 7 * kChunk, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = launch_first_hits(a, st);
        if (e == cudaSuccess) e = launch_first_finalize(a, keys, E->entry + 7 * first, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->h_counters, c->counters, kNumCounters * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st);
    // the scratch buffers are released once the stream has consumed them
    cudaError_t se = cudaStreamSynchronize(st);
    ctx_free(c, rgb);
    ctx_free(c, keys);
    if (e == cudaSuccess) e = se;
    if (e != cudaSuccess) {
        cvs_etab_destroy(E);
        return fail(e == cudaErrorMemoryAllocation ? CVS_ERR_NO_MEMORY : CVS_ERR_CUDA,
                    "cvs_etab_build: %s", cudaGetErrorString(e));
    }
    c->last = cvs_stats{};
    c->last.candidates = kColours * (int64_t)c->grid.K * c->grid.N;
    c->last.targets = kColours;
    c->last.symmetric = c->grid.sym;
    c->last.precision = (int32_t)prec;
    c->last_pending = true;
    collect_stats(c);
    *out = E;
    return CVS_OK;
}

void cvs_etab_destroy(cvs_etab* E) {
    if (!E) return;
    cudaSetDevice(E->device);
    cudaDeviceSynchronize();
    if (E->entry) cudaFree(E->entry);
    delete E;
}

cvs_status cvs_etab_embed_image(cvs_etab* E, const cvs_image* img, const uint8_t* pattern_dev,
                                int64_t pattern_pitch, uint8_t* frame_a_dev, uint8_t* frame_b_dev,
                                int64_t frame_pitch, uint32_t* choice_dev, void* stream) {
    if (!E || !img || !pattern_dev || !frame_a_dev || !frame_b_dev)
        return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (!img->rgb || img->width <= 0 || img->height <= 0 || img->pitch_bytes < 3LL * img->width)
        return fail(CVS_ERR_INVALID_ARG, "bad image pointer, size or pitch");
    if (pattern_pitch < img->width) return fail(CVS_ERR_INVALID_ARG, "pattern pitch < width");
    if (frame_pitch < 3LL * img->width) return fail(CVS_ERR_INVALID_ARG, "frame pitch < 3 * width");
    if (frame_a_dev == frame_b_dev) return fail(CVS_ERR_INVALID_ARG, "the two frames must differ");
    if ((int64_t)img->width * img->height >= ((int64_t)1 << 40))
        return fail(CVS_ERR_INVALID_ARG, "image too large");
    CVS_CUDA(cudaSetDevice(E->device));
    CVS_CUDA(launch_etab_gather(E->entry, img->rgb, img->pitch_bytes, img->width, img->height,
                                pattern_dev, pattern_pitch, frame_a_dev, frame_b_dev, frame_pitch,
                                choice_dev, (cudaStream_t)stream));
    return CVS_OK;
}

cvs_status cvs_reserve(cvs_ctx* c, const cvs_grid* grid, int64_t max_targets, int32_t max_images) {
    if (!c) return fail(CVS_ERR_INVALID_ARG, "NULL context");
    if (max_targets < 0 || max_images < 0) return fail(CVS_ERR_INVALID_ARG, "negative size");
    cvs_status st0 = grid ? check_grid(grid) : CVS_OK;
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK && grid) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK && max_targets > 0) st0 = ensure_targets(c, max_targets);
    // an image batch this large may take the per-batch de-duplication
    if (st0 == CVS_OK && c->dedup == 2 && max_targets >= kDedupAutoPixels &&
        ensure_dedup(c) != CVS_OK) {  // beyond the budget: such batches search per pixel
        drop_dedup(c);
        g_err.clear();
    }
    if (st0 != CVS_OK) return st0;
    if (max_images > 0) CVS_TRY(grow(c, &c->d_imgs, &c->cap_imgs, max_images));
    return CVS_OK;
}

cvs_status cvs_synchronize(cvs_ctx* c, void* stream) {
    if (!c) return fail(CVS_ERR_INVALID_ARG, "NULL context");
    cvs_status st0 = set_device(c);
    if (st0 != CVS_OK) return st0;
    CVS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    CVS_CUDA(cudaStreamSynchronize(c->own));
    collect_stats(c);
    return CVS_OK;
}

cvs_status cvs_get_stats(cvs_ctx* c, cvs_stats* out) {
    if (!c || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (c->last_pending) return fail(CVS_ERR_INVALID_ARG, "last search not synchronised yet");
    *out = c->last;
    return CVS_OK;
}

cvs_status cvs_precision_probe(cvs_ctx* c, const uint8_t* rgb_dev, int64_t n,
                               const cvs_grid* grid, cvs_precision_report* out) {
    if (!c || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n <= 0 || !rgb_dev) return fail(CVS_ERR_INVALID_ARG, "need n > 0 colours");
    cvs_status st0 = check_grid(grid);
    if (st0 == CVS_OK) st0 = set_device(c);
    if (st0 == CVS_OK) st0 = ensure_grid(c, grid);
    if (st0 == CVS_OK) st0 = ensure_targets(c, n);
    if (st0 != CVS_OK) return st0;
    cudaStream_t st = c->own;
    // d_probe: three float maxima, a pad word, then three 64-bit counts
    CVS_CUDA(cudaMemsetAsync(c->d_probe, 0, 40, st));
    CVS_CUDA(launch_setup_colors(rgb_dev, n, c->grid.rmax, c->tf, c->td, c->acc, st));
    CVS_CUDA(launch_precision_probe(c->tf, c->td, n, c->grid, c->qkey, (float)(0.5 - c->window),
                                    c->d_probe, c->d_probe + 1, c->d_probe + 2,
                                    reinterpret_cast<unsigned long long*>(c->d_probe + 4),
                                    c->num_sms, st));
    unsigned int h[10] = {};
    CVS_CUDA(cudaMemcpyAsync(h, c->d_probe, 40, cudaMemcpyDeviceToHost, st));
    CVS_CUDA(cudaStreamSynchronize(st));
    float fv, fl, fa;
    std::memcpy(&fv, &h[0], 4);
    std::memcpy(&fl, &h[1], 4);
    std::memcpy(&fa, &h[2], 4);
    unsigned long long cnt[3];
    std::memcpy(cnt, &h[4], 24);
    out->max_code_err = fv;
    out->max_lin_err = fl;
    out->max_lab_err = fa;
    out->n_wrong_codes = (int64_t)cnt[0];
    out->n_unflagged_wrong = (int64_t)cnt[1];
    out->n_values = (int64_t)cnt[2];
    out->window = c->window;
    return CVS_OK;
}

}  // extern "C"
