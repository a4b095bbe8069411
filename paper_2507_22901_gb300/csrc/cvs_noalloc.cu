// cvs_noalloc.cu - cvs_search_colors_noalloc: the per-colour search for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc: code hosted inside an application whose
// own memory manager owns the device heap and rejects outside allocations, or a
// latency-critical loop in which cudaMalloc's implicit device synchronisation
// would stall every other stream.  This entry point needs no context and makes
// no allocation: every scratch buffer of the search (grid tables, threshold
// keys, work counters, per-target constants and accumulators) is carved out of
// one fixed array of this library, g_noalloc_scratch, which every GPU that loads
// the library holds until the process exits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "cvs_internal.h"
#include "cvs_tables.h"

namespace {

constexpr int64_t kMaxTargets = 4096;
constexpr int32_t kMaxRadii = 1024;
constexpr int32_t kMaxAngles = 1024;
constexpr size_t kScratchBytes = 512 * 1024;

constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the buffers inside the scratch array.
constexpr size_t kOffQkey = 0;
constexpr size_t kOffCounters = kOffQkey + up256(257 * sizeof(long long));
constexpr size_t kOffStatus = kOffCounters + up256(cvs::kNumCounters * sizeof(unsigned long long));
constexpr size_t kOffR32 = kOffStatus + up256(sizeof(int));
constexpr size_t kOffSc32 = kOffR32 + up256(kMaxRadii * sizeof(float));
constexpr size_t kOffR64 = kOffSc32 + up256(kMaxAngles * sizeof(float2));
constexpr size_t kOffS64 = kOffR64 + up256(kMaxRadii * sizeof(double));
constexpr size_t kOffC64 = kOffS64 + up256(kMaxAngles * sizeof(double));
constexpr size_t kOffAngles = kOffC64 + up256(kMaxAngles * sizeof(double));
constexpr size_t kOffTf = kOffAngles + up256(kMaxAngles * sizeof(double));
constexpr size_t kTfBytes = 48, kTdBytes = 32;  // sizes of TargetF32 / TargetF64
constexpr size_t kOffTd = kOffTf + up256(kMaxTargets * kTfBytes);
constexpr size_t kOffAcc = kOffTd + up256(kMaxTargets * kTdBytes);
constexpr size_t kEnd = kOffAcc + up256(kMaxTargets * sizeof(cvs::Acc));
static_assert(kEnd <= kScratchBytes, "no-alloc scratch layout exceeds the array");

// The scratch array.  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mu;

thread_local char g_msg[256];

cvs_status fail(cvs_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    cvs::set_error_message(g_msg);
    return st;
}

long long host_dkey(double x) {
    long long k;
    std::memcpy(&k, &x, sizeof k);
    return k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// The 257 quantisation threshold keys, formed once on the host; static, so the
// source of every call's asynchronous copy outlives the copy.
struct QKeys {
    long long v[257];
    QKeys() {
        const double thr[257] = CVS_QTHR_INIT;
        for (int i = 0; i < 257; ++i) v[i] = host_dkey(thr[i]);
    }
};
const QKeys g_qkeys;

// Once per device, with that device current: the scratch array's device
// address.  (A cudaDeviceReset between calls would invalidate the cached
// address; the entry point does not support that.)
cvs_status device_setup(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch_ptr[device]) {
        *out = g_scratch_ptr[device];
        return CVS_OK;
    }
    if (cvs::target_f32_size() != kTfBytes || cvs::target_f64_size() != kTdBytes)
        return fail(CVS_ERR_CUDA, "no-alloc scratch layout does not match the target records");
    unsigned char* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(CVS_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch): %s",
                    cudaGetErrorString(e));
    g_scratch_ptr[device] = p;
    *out = p;
    return CVS_OK;
}

cvs_status run(int device, const uint8_t* rgb_dev, int64_t n, const cvs_grid* g,
               const cvs_thresholds* thr, cvs_precision prec, const cvs_capacity_map* out,
               cudaStream_t st) {
    unsigned char* p = nullptr;
    cvs_status s = device_setup(device, &p);
    if (s != CVS_OK) return s;
#define NA_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return fail(CVS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
    const int K = g->n_radii, N = g->n_angles;
    cvs::GridDev d;
    d.K = K;
    d.N = N;
    d.r32 = reinterpret_cast<float*>(p + kOffR32);
    d.sc32 = reinterpret_cast<float2*>(p + kOffSc32);
    d.r64 = reinterpret_cast<double*>(p + kOffR64);
    d.s64 = reinterpret_cast<double*>(p + kOffS64);
    d.c64 = reinterpret_cast<double*>(p + kOffC64);
    int* status = reinterpret_cast<int*>(p + kOffStatus);
    double* angles = reinterpret_cast<double*>(p + kOffAngles);
    float r32[kMaxRadii];
    double sh[kMaxAngles], ch[kMaxAngles];
    double rmax = 0.0;
    for (int i = 0; i < K; ++i) {
        r32[i] = (float)g->radii[i];
        if (g->radii[i] > rmax) rmax = g->radii[i];
    }
    d.rmax = rmax;
    // every call writes all it reads: the threshold keys, then the grid
    NA_CUDA(cudaMemcpyAsync(p + kOffQkey, g_qkeys.v, sizeof g_qkeys.v, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemcpyAsync(d.r64, g->radii, sizeof(double) * K, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemcpyAsync(d.r32, r32, sizeof(float) * K, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemcpyAsync(angles, g->angles_deg, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    NA_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    NA_CUDA(cvs::launch_trig_table(angles, N, d.s64, d.c64, d.sc32, status, st));
    int hstatus = 0;
    NA_CUDA(cudaMemcpyAsync(sh, d.s64, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaMemcpyAsync(ch, d.c64, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (hstatus) return fail(CVS_ERR_NUMERIC, "an angle's sine could not be certified");
    const int sym = cvs::fold_by_180(sh, ch, N);
    d.sym = sym;
    d.H = sym ? N / 2 : N;
    if (n == 0) return CVS_OK;

    auto* tf = reinterpret_cast<cvs::TargetF32*>(p + kOffTf);
    auto* td = reinterpret_cast<cvs::TargetF64*>(p + kOffTd);
    auto* acc = reinterpret_cast<cvs::Acc*>(p + kOffAcc);
    auto* counters = reinterpret_cast<unsigned long long*>(p + kOffCounters);
    int num_sms = 0;
    NA_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    cvs::SearchArgs a{};
    a.tf = tf;
    a.td = td;
    a.acc = acc;
    a.n_targets = n;
    a.grid = d;
    a.qkey = reinterpret_cast<const long long*>(p + kOffQkey);
    s = cvs_signal_bounds(thr, &a.hi_min, &a.lo_max);
    if (s != CVS_OK) return s;
    a.mask2 = thr->pattern_mask << 1;
    a.clip = thr->gamut_mode;
    a.half_w = (float)(0.5 - 2e-3);
    a.prec = (int32_t)prec;
    a.list_mode = 0;
    a.work_counter = counters;
    a.stats = counters + 1;
    a.shape.block = cvs::kSearchBlock;
    a.shape.blocks_per_sm = 0;
    a.shape.kchunk = cvs::auto_kchunk(num_sms, n, K, d.H);
    a.num_sms = num_sms;
    NA_CUDA(cvs::launch_setup_colors(rgb_dev, n, rmax, tf, td, acc, st));
    NA_CUDA(cudaMemsetAsync(counters, 0, cvs::kNumCounters * sizeof(unsigned long long), st));
    NA_CUDA(cvs::launch_search(a, st));
    NA_CUDA(cvs::launch_finalize_colors(acc, n, out->max_r, out->count, out->pmask, st));
    return CVS_OK;
#undef NA_CUDA
}

}  // namespace

extern "C" cvs_status cvs_search_colors_noalloc(int device, const uint8_t* rgb_dev, int64_t n,
                                                const cvs_grid* grid, const cvs_thresholds* thr,
                                                cvs_precision prec, const cvs_capacity_map* out,
                                                void* stream) {
    if (!grid || !thr || !out) return fail(CVS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > kMaxTargets)
        return fail(CVS_ERR_INVALID_ARG,
                    "cvs_search_colors_noalloc: n = %lld colours, the fixed scratch holds at most %lld",
                    (long long)n, (long long)kMaxTargets);
    if (n > 0 && (!rgb_dev || !out->max_r || !out->count || !out->pmask))
        return fail(CVS_ERR_INVALID_ARG, "NULL device buffer");
    if (!grid->radii || !grid->angles_deg || grid->n_radii <= 0 || grid->n_angles <= 0)
        return fail(CVS_ERR_INVALID_ARG, "empty or NULL grid");
    if (grid->n_radii > kMaxRadii || grid->n_angles > kMaxAngles)
        return fail(CVS_ERR_INVALID_ARG,
                    "cvs_search_colors_noalloc: grid %d x %d exceeds the fixed scratch limit %d x %d",
                    grid->n_radii, grid->n_angles, kMaxRadii, kMaxAngles);
    for (int i = 0; i < grid->n_radii; ++i)
        if (!std::isfinite(grid->radii[i]) || grid->radii[i] < 0.0 || grid->radii[i] > cvs::kMaxRadius)
            return fail(CVS_ERR_INVALID_ARG, "radius %d must be in [0, %g]", i, cvs::kMaxRadius);
    for (int i = 0; i < grid->n_angles; ++i)
        if (!std::isfinite(grid->angles_deg[i]))
            return fail(CVS_ERR_INVALID_ARG, "angle %d is not finite", i);
    if (prec != CVS_PREC_FP32_RECHECK && prec != CVS_PREC_FP64)
        return fail(CVS_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (prec == CVS_PREC_FP32_RECHECK)
        for (int i = 0; i < grid->n_radii; ++i)
            if (grid->radii[i] > cvs::kFp32MaxRadius)
                return fail(CVS_ERR_INVALID_ARG,
                            "CVS_PREC_FP32_RECHECK is validated for radii up to %g (radius %d is "
                            "%g): pass CVS_PREC_FP64", cvs::kFp32MaxRadius, i, grid->radii[i]);
    int32_t hi, lo;
    cvs_status s = cvs_signal_bounds(thr, &hi, &lo);  // validates the thresholds
    if (s != CVS_OK) return s;
    if (thr->max_dl > 0.0 && std::isfinite(thr->max_dl))
        return fail(CVS_ERR_INVALID_ARG,
                    "cvs_search_colors_noalloc: the luminance limit max_dl needs a 128 MiB table "
                    "of L* values that the fixed scratch cannot hold; pass max_dl = 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
        device >= kMaxDevices)
        return fail(CVS_ERR_INVALID_ARG, "device %d is not available", device);
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = device;
    if (cudaSetDevice(device) != cudaSuccess)
        return fail(CVS_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    s = run(device, rgb_dev, n, grid, thr, prec, out, (cudaStream_t)stream);
    cudaSetDevice(prev);
    return s;
}
