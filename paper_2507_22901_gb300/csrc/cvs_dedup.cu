// cvs_dedup.cu - per-batch colour de-duplication for the image search (sm_103a).
//
// A pixel's maps are a pure function of its colour (and of the grid and
// thresholds), so a batch of images needs one search per distinct colour:
//   mark   : every pixel sets its colour's byte in a 2^24-entry presence map;
//   scan   : an exclusive scan of the map gives each present colour its index
//            among the distinct colours and lists them in colour order;
//   search : the regular per-colour search over the distinct colours;
//   gather : every pixel reads its colour's accumulator into its maps.
// The scan is three kernels: per-block sums of 16,384 entries, a scan of the
// 1,024 block sums, then per-thread rescans that write the indices.
#include <cuda_runtime.h>

#include "cvs_internal.h"

namespace cvs {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 16;
constexpr int kScanPerBlock = kScanThreads * kScanPerThread;  // 16,384
constexpr int kScanBlocks = (1 << 24) / kScanPerBlock;       // 1,024

__device__ __forceinline__ int find_image_d(const ImageDesc* imgs, int n_imgs, int64_t p) {
    int lo = 0, hi = n_imgs - 1;  // largest i with imgs[i].first <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].first <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t pixel_colour(const ImageDesc* imgs, int n_imgs, int64_t p,
                                                 int& img, int64_t& local) {
    img = find_image_d(imgs, n_imgs, p);
    const ImageDesc& im = imgs[img];
    local = p - im.first;
    const int64_t y = local / im.width, x = local - y * im.width;
    const uint8_t* px = im.rgb + y * im.pitch + 3 * x;
    return ((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | px[2];
}

__global__ void k_mark_colours(const ImageDesc* __restrict__ imgs, int n_imgs, int64_t total,
                               uint8_t* __restrict__ present) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        int img;
        int64_t local;
        present[pixel_colour(imgs, n_imgs, p, img, local)] = 1;
    }
}

// Exclusive scan of a block's thread sums; returns the thread's offset and
// writes the block total to *total (thread 0).
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, off);
            if (lane >= off) w += y;
        }
        warp_sums[lane] = w;  // inclusive over warps
        if (lane == 31) *total = w;
    }
    __syncthreads();
    const int before_warp = warp > 0 ? warp_sums[warp - 1] : 0;
    return before_warp + x - v;
}

__device__ __forceinline__ int thread_count(const uint8_t* present, int64_t base) {
    const uint4 q = *reinterpret_cast<const uint4*>(present + base);  // 16 bytes
    return __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);     // bytes are 0 or 1
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const uint8_t* __restrict__ present,
                                                            int* __restrict__ block_sums) {
    __shared__ int warp_sums[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + (int64_t)threadIdx.x * kScanPerThread;
    block_exclusive_scan(thread_count(present, base), warp_sums, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the kScanBlocks block sums (in place); the
// grand total goes to *n_unique.
__global__ void __launch_bounds__(kScanThreads) k_scan_block_sums(int* __restrict__ block_sums,
                                                                  int* __restrict__ n_unique) {
    __shared__ int warp_sums[32];
    __shared__ int total;
    const int v = block_sums[threadIdx.x];
    const int ex = block_exclusive_scan(v, warp_sums, &total);
    block_sums[threadIdx.x] = ex;
    if (threadIdx.x == 0) *n_unique = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_finish(const uint8_t* __restrict__ present,
                                                              const int* __restrict__ block_offs,
                                                              int32_t* __restrict__ index,
                                                              uint8_t* __restrict__ unique_rgb) {
    __shared__ int warp_sums[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + (int64_t)threadIdx.x * kScanPerThread;
    int u = block_offs[blockIdx.x] +
            block_exclusive_scan(thread_count(present, base), warp_sums, &total);
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        const int64_t c = base + j;
        if (present[c]) {
            index[c] = u;
            unique_rgb[3 * (int64_t)u] = (uint8_t)(c >> 16);
            unique_rgb[3 * (int64_t)u + 1] = (uint8_t)(c >> 8);
            unique_rgb[3 * (int64_t)u + 2] = (uint8_t)c;
            ++u;
        }
    }
}

__global__ void k_dedup_gather(const ImageDesc* __restrict__ imgs, int n_imgs, int64_t total,
                               const int32_t* __restrict__ index, const Acc* __restrict__ acc) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        int img;
        int64_t local;
        const uint32_t c = pixel_colour(imgs, n_imgs, p, img, local);
        const Acc a = acc[index[c]];
        const ImageDesc& im = imgs[img];
        im.max_r[local] = __int_as_float(a.rmax_bits);
        im.count[local] = a.count;
        im.pmask[local] = (uint8_t)a.pmask;
    }
}

int grid_for(int64_t n, int threads) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads, cap = (int64_t)(sms > 0 ? sms : 1) * 32;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_dedup_mark(const ImageDesc* imgs, int n_imgs, int64_t total, uint8_t* present,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(present, 0, (size_t)1 << 24, st);
    if (e != cudaSuccess || total <= 0) return e;
    k_mark_colours<<<grid_for(total, 256), 256, 0, st>>>(imgs, n_imgs, total, present);
    return cudaGetLastError();
}

cudaError_t launch_dedup_scan(const uint8_t* present, int* block_sums, int* n_unique,
                              int32_t* index, uint8_t* unique_rgb, cudaStream_t st) {
    k_scan_sums<<<kScanBlocks, kScanThreads, 0, st>>>(present, block_sums);
    k_scan_block_sums<<<1, kScanThreads, 0, st>>>(block_sums, n_unique);
    k_scan_finish<<<kScanBlocks, kScanThreads, 0, st>>>(present, block_sums, index, unique_rgb);
    return cudaGetLastError();
}

cudaError_t launch_dedup_gather(const ImageDesc* imgs, int n_imgs, int64_t total,
                                const int32_t* index, const Acc* acc, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    k_dedup_gather<<<grid_for(total, 256), 256, 0, st>>>(imgs, n_imgs, total, index, acc);
    return cudaGetLastError();
}

}  // namespace cvs
