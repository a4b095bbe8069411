// cvs_embed.cu - the embedding step (Fig. 1a) on sm_103a.
//
// A display shows two frames in alternation; where a pixel carries
// information, the frames hold the two colours of a point-symmetric pair that
// passes the embedding-signal condition with the requested 3-bit pattern, so
// a person sees the pixel's own colour and a camera sees the channels that
// switch.  Per pixel the pair is the first passing candidate of that pattern
// in (radius value, radius index k, angle index m) order: the smallest shift
// in L*a*b*, then the caller's order.
//
// One warp per pixel (persistent warps over an atomic pixel counter) walks
// the radii in increasing order and stops at the first radius with a hit.
// Within a radius, lanes take angle slots 32 at a time through the FP32 slot
// of cvs_slot32.cuh; flagged slots are only decided (exact interval analysis,
// FP64 where that cannot decide) when their angle index lies below the best
// unflagged hit.  A winner whose codes are uncertain gets its codes in FP64.
#include <cuda_runtime.h>

#include "cvs_device.cuh"
#include "cvs_internal.h"
#include "cvs_slot32.cuh"

namespace cvs {

namespace {

constexpr uint32_t kNoChoice = 0xFFFFFFFFu;
constexpr int kNone = 0x7FFFFFFF;

template <bool CLIP>
__device__ __forceinline__ void codes64_slot(const EmbedArgs& A, const TargetF64& D, int k, int h,
                                             int qp[3], int qm[3]) {
    pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + k), __ldg(A.grid.s64 + h),
                 __ldg(A.grid.c64 + h), A.qkey, qp, qm);
    if (CLIP) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            qp[c] = min(max(qp[c], 0), 255);
            qm[c] = min(max(qm[c], 0), 255);
        }
    }
}

// Exact decision of one slot in FP64 (the codes come back clamped in clip mode).
template <bool CLIP>
__device__ __forceinline__ int decide64(const EmbedArgs& A, const TargetF64& D, int k, int h,
                                        int qp[3], int qm[3]) {
    codes64_slot<CLIP>(A, D, k, h, qp, qm);
    Decide dc{A.hi_min, A.lo_max, A.mask2, CLIP ? 1 : 0};
    return decide_codes(qp, qm, dc);
}

// Per lane: the smallest angle slot of radius k (among this lane's slots)
// whose pair passes with pattern p, and that pair's codes.
struct Hit {
    int h;
    int qp[3], qm[3];
    bool exact;  // false: the decision is exact but the codes may be one off
};

__device__ __forceinline__ void take(Hit& w, int h, const int qp[3], const int qm[3],
                                     bool exact) {
    w.h = h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        w.qp[c] = qp[c];
        w.qm[c] = qm[c];
    }
    w.exact = exact;
}

// One flagged FP32 slot: exact pattern by interval analysis, FP64 where the
// bounds cannot decide.  Records a hit of pattern p in w.
template <bool FAST, bool CLIP>
__device__ __forceinline__ void decide_flagged(const EmbedArgs& A, const TargetF32& T,
                                               const ChainF32& C, const TargetF64& D, float2 r2,
                                               float4 sc, int k, int h, int p, Hit& w,
                                               unsigned long long& n_exact,
                                               unsigned long long& n_re) {
    const Intervals I = intervals32<FAST>(T, C, r2, sc, A.half_w, CLIP ? 1 : 0);
    const int pc = certain_from(I, A.hi_min, A.lo_max, A.mask2, CLIP ? 1 : 0, 0);
    ++n_exact;
    if (pc == p) {
        take(w, h, I.lo, I.lo + 3, !I.any_flag);  // lo == hi for every unflagged code
    } else if (pc < 0) {
        int qp[3], qm[3];
        ++n_re;
        if (decide64<CLIP>(A, D, k, h, qp, qm) == p) take(w, h, qp, qm, true);
    }
}

// Radius k of one pixel: returns the smallest passing angle slot of pattern p
// over the warp (kNone if none; warp-uniform); the lane holding it has it in w.
template <int PREC, bool FAST, bool CLIP>
__device__ __forceinline__ int embed_radius(const EmbedArgs& A, const float2* r2s,
                                            const float4* sc4s, const uint8_t* lut,
                                            const TargetF32& T, const PairsT& P,
                                            const PairsC& PC, const ChainF32& C,
                                            const TargetF64& D, int k, int p, Hit& w,
                                            unsigned long long& n_exact,
                                            unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    const float2 r2 = r2s[k];
    w.h = kNone;
    if (PREC == CVS_PREC_FP32_RECHECK) {
        const bool pow_only = FAST && pow_branch_only(T, C, r2.x);
        uint64_t fbits = 0;  // iterations (below 64) whose slot of this lane was flagged
        for (int it = 0; it * 32 < H; ++it) {
            const int h = it * 32 + (int)lane;
            const bool active = h < H && w.h == kNone;
            const float4 sc = sc4s[h < H ? h : 0];
            const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y)), w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
            int yp[3], ym[3];
            bool flag;
            if (pow_only) flag = codes32<FAST, false>(P, PC, u2, w2, A.half_w, yp, ym);
            else flag = codes32<FAST, true>(P, PC, u2, w2, A.half_w, yp, ym);
            const int pat = decide32<CLIP>(yp, ym, lut, A.mask2);
            if (active) {
                if (!flag) {
                    if (pat == p) {
                        int qp[3], qm[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            qp[c] = yp[c] - kMagicBits;
                            qm[c] = ym[c] - kMagicBits;
                            if (CLIP) {
                                qp[c] = min(max(qp[c], 0), 255);
                                qm[c] = min(max(qm[c], 0), 255);
                            }
                        }
                        take(w, h, qp, qm, true);
                    }
                } else if (it < 64) {
                    fbits |= 1ull << it;
                } else {  // more than 2048 slots per radius: decide in place
                    decide_flagged<FAST, CLIP>(A, T, C, D, r2, sc, k, h, p, w, n_exact, n_re);
                }
            }
        }
        // flagged slots matter only below the warp's best unflagged hit
        const int best0 = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)w.h);
        if (best0 != kNone) {
            const int lim = best0 - (int)lane;  // slot it * 32 + lane < best0
            const int n_ok = lim <= 0 ? 0 : (lim + 31) >> 5;
            fbits &= n_ok >= 64 ? ~0ull : ((1ull << n_ok) - 1ull);
        }
        while (__any_sync(0xFFFFFFFFu, fbits != 0ull)) {
            if (fbits) {
                const int it = __ffsll((long long)fbits) - 1;
                fbits &= fbits - 1ull;
                const int h = it * 32 + (int)lane;
                if (h < w.h)  // a lane's earlier hit beats its later slots
                    decide_flagged<FAST, CLIP>(A, T, C, D, r2, sc4s[h], k, h, p, w, n_exact, n_re);
                else
                    fbits = 0ull;
            }
        }
    } else {
        for (int it = 0; it * 32 < H; ++it) {
            const int h = it * 32 + (int)lane;
            if (h < H && w.h == kNone) {
                int qp[3], qm[3];
                if (decide64<CLIP>(A, D, k, h, qp, qm) == p) take(w, h, qp, qm, true);
            }
        }
    }
    return (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)w.h);
}

// One pixel with requested pattern p: radii in increasing order until a hit;
// the winning lane writes both frames and the choice.  Returns true on a hit.
template <int PREC, bool FAST, bool CLIP>
__device__ __forceinline__ bool embed_pixel(const EmbedArgs& A, const float2* r2s,
                                            const float4* sc4s, const uint8_t* lut,
                                            const PairsC& PC, const ChainF32& C, int64_t t,
                                            uint8_t* fa, uint8_t* fb, int p,
                                            unsigned long long& n_exact,
                                            unsigned long long& n_re) {
    TargetF32 T{};
    if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
    const TargetF64 D = A.td[t];
    const PairsT P = make_pairs(T);
    for (int kk = 0; kk < A.grid.K; ++kk) {
        const int k = __ldg(A.order + kk);
        Hit w;
        const int best = embed_radius<PREC, FAST, CLIP>(A, r2s, sc4s, lut, T, P, PC, C, D, k, p, w,
                                                        n_exact, n_re);
        if (best == kNone) continue;
        if (w.h == best) {
            if (!w.exact) codes64_slot<CLIP>(A, D, k, best, w.qp, w.qm);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                fa[c] = (uint8_t)w.qp[c];
                fb[c] = (uint8_t)w.qm[c];
            }
            if (A.choice) A.choice[t] = (uint32_t)k | ((uint32_t)best << 16);
        }
        return true;
    }
    return false;
}

template <int PREC, bool CLIP>
__global__ void __launch_bounds__(kSearchBlock) k_embed(const EmbedArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H;
    float2* r2s = reinterpret_cast<float2*>(smem);
    float4* sc4s = reinterpret_cast<float4*>(smem + ((K * 8 + 15) & ~15));
    uint8_t* lut = smem + ((K * 8 + 15) & ~15) + H * 16;
    build_decide_lut(lut, A.hi_min, A.lo_max);
    for (int i = threadIdx.x; i < K; i += blockDim.x) r2s[i] = dup(A.grid.r32[i]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        const float2 sc = A.grid.sc32[i];
        sc4s[i] = make_float4(sc.x, -sc.x, sc.y, -sc.y);
    }
    __syncthreads();
    ChainF32 C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C.Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        C.Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    const PairsC PC = make_pairs(C);
    const unsigned lane = lane_id();
    unsigned long long n_exact = 0, n_re = 0;
    while (true) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(A.work_counter, 1ull);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= (unsigned long long)A.n) break;
        const int64_t t = (int64_t)item;
        const int64_t y = t / A.width, x = t - y * A.width;
        const uint8_t* src = A.rgb + y * A.pitch + 3 * x;
        uint8_t* fa = A.frame_a + y * A.frame_pitch + 3 * x;
        uint8_t* fb = A.frame_b + y * A.frame_pitch + 3 * x;
        const int p = A.pattern[y * A.pattern_pitch + x];
        bool hit = false;
        if (p >= 1 && p <= 7) {
            if (PREC == CVS_PREC_FP32_RECHECK && (A.tf[t].flags & 1u))
                hit = embed_pixel<PREC, true, CLIP>(A, r2s, sc4s, lut, PC, C, t, fa, fb, p, n_exact,
                                                    n_re);
            else
                hit = embed_pixel<PREC, false, CLIP>(A, r2s, sc4s, lut, PC, C, t, fa, fb, p,
                                                     n_exact, n_re);
        }
        if (!hit && lane == 0) {
            const uint8_t r = src[0], g = src[1], b = src[2];
            fa[0] = r; fa[1] = g; fa[2] = b;
            fb[0] = r; fb[1] = g; fb[2] = b;
            if (A.choice) A.choice[t] = kNoChoice;
        }
        __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n_exact += __shfl_xor_sync(0xFFFFFFFFu, n_exact, off);
        n_re += __shfl_xor_sync(0xFFFFFFFFu, n_re, off);
    }
    if (lane == 0) {
        if (n_exact) atomicAdd(A.stats + 0, n_exact);
        if (n_re) atomicAdd(A.stats + 1, n_re);
    }
}

int embed_smem_bytes(const GridDev& g) { return ((g.K * 8 + 15) & ~15) + g.H * 16 + 3 * 512; }

template <int PREC, bool CLIP>
cudaError_t launch_embed_t(const EmbedArgs& a, cudaStream_t st) {
    const int smem = embed_smem_bytes(a.grid);
    const void* fn = (const void*)k_embed<PREC, CLIP>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSearchBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_embed<PREC, CLIP><<<a.num_sms * per_sm, kSearchBlock, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_embed(const EmbedArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    if (a.prec == CVS_PREC_FP64)
        return a.clip ? launch_embed_t<CVS_PREC_FP64, true>(a, st)
                      : launch_embed_t<CVS_PREC_FP64, false>(a, st);
    return a.clip ? launch_embed_t<CVS_PREC_FP32_RECHECK, true>(a, st)
                  : launch_embed_t<CVS_PREC_FP32_RECHECK, false>(a, st);
}

}  // namespace cvs
