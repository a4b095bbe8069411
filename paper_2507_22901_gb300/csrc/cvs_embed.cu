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

// The luminance limit (when on) on a pair of exact codes.
__device__ __forceinline__ bool dl_pass(const EmbedArgs& A, const TargetF64& D, const int qp[3],
                                        const int qm[3]) {
    return !A.ltab || dl_ok(A.ltab, A.max_dl, D.L, qp, qm);
}

// One flagged FP32 slot: exact pattern by interval analysis, FP64 where the
// bounds cannot decide (or, under the luminance limit, where a passing pair's
// codes are not all certain).  Records a hit of pattern p in w.
template <bool FAST, bool CLIP>
__device__ __forceinline__ void decide_flagged(const EmbedArgs& A, const TargetF32& T,
                                               const ChainF32& C, const TargetF64& D, float2 r2,
                                               float4 sc, int k, int h, int p, Hit& w,
                                               unsigned long long& n_exact,
                                               unsigned long long& n_re) {
    const Intervals I = intervals32<FAST>(T, C, r2, sc, A.half_w, CLIP ? 1 : 0);
    const int pc = certain_from(I, A.hi_min, A.lo_max, A.mask2, CLIP ? 1 : 0, A.ltab ? 1 : 0);
    ++n_exact;
    if (pc == p) {
        if (dl_pass(A, D, I.lo, I.lo + 3))
            take(w, h, I.lo, I.lo + 3, !I.any_flag);  // lo == hi for every unflagged code
    } else if (pc < 0) {
        int qp[3], qm[3];
        ++n_re;
        if (decide64<CLIP>(A, D, k, h, qp, qm) == p && dl_pass(A, D, qp, qm))
            take(w, h, qp, qm, true);
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
            float2 lin[3];
            lin32<FAST>(P, PC, u2, w2, lin);
            // gamut reject: 32 slots that all leave the gamut hold no hit
            if (!CLIP && __all_sync(0xFFFFFFFFu, !active || surely_out32(lin))) continue;
            int yp[3], ym[3];
            bool flag;
            if (pow_only) flag = encode32<false>(lin, A.half_w, yp, ym, nullptr);
            else flag = encode32<true>(lin, A.half_w, yp, ym, nullptr);
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
                        if (dl_pass(A, D, qp, qm)) take(w, h, qp, qm, true);
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
                if (decide64<CLIP>(A, D, k, h, qp, qm) == p && dl_pass(A, D, qp, qm))
                    take(w, h, qp, qm, true);
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
    const uint32_t need = (uint32_t)p;  // channels pattern p needs high (bit 2 - c)
    // a channel p needs high that cannot be high at the largest radius: no pair
    if (PREC == CVS_PREC_FP32_RECHECK && FAST &&
        (high_possible(T, C, r2s[__ldg(A.order + A.grid.K - 1)].x, A.hi_min) & need) != need)
        return false;
    for (int kk = 0; kk < A.grid.K; ++kk) {
        const int k = __ldg(A.order + kk);
        // at this radius a channel p needs high cannot be high
        if (PREC == CVS_PREC_FP32_RECHECK && FAST &&
            (high_possible(T, C, r2s[k].x, A.hi_min) & need) != need)
            continue;
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

// ------------------------------------------------------------ embedding table
// A pixel's pair depends only on its colour and requested pattern, so a table
// over all 2^24 colours x 7 patterns turns the embedding of any frame into a
// gather.  The build is one search of every colour that keeps, per pattern,
// the first hit in (rank of the radius in sorted order, angle slot) order:
// key = rank << 16 | h.  Unflagged passes enter through a warp-wide OR of the
// patterns seen (new patterns take the lowest lane, i.e. the smallest key of
// the iteration); flagged slots are marked in a per-lane bitmap and decided
// after each segment, entering through atomicMin on the key.
constexpr int kHitWords = 8;
constexpr int kHitSegIters = 32 * kHitWords;

// Flagged slots of one segment: exact decision, atomicMin of passing keys.
template <int PREC, bool FAST, bool CLIP>
__device__ __forceinline__ void first_flagged(const FirstHitArgs& A, const float2* r2s,
                                              const float4* sc4s, const TargetF32& T,
                                              const ChainF32& C, const TargetF64& D, int64_t t,
                                              int kk0, int seg0, int nwords, uint32_t* fb,
                                              unsigned long long& n_exact,
                                              unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    for (int w = 0; w < nwords; ++w) {
        uint32_t bits = fb[w * 32 + lane];
        fb[w * 32 + lane] = 0u;
        while (__any_sync(0xFFFFFFFFu, bits != 0u)) {
            if (bits) {
                const int j = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int i = (seg0 + 32 * w + j) * 32 + (int)lane;
                const int dk = i / H;
                const int kq = kk0 + dk, hq = i - dk * H;
                const Intervals I = intervals32<FAST>(T, C, r2s[kq], sc4s[hq], A.half_w, CLIP ? 1 : 0);
                // under the luminance limit a pass needs certain codes
                int pc = certain_from(I, A.hi_min, A.lo_max, A.mask2, CLIP ? 1 : 0, A.ltab ? 1 : 0);
                ++n_exact;
                if (pc > 0 && A.ltab && !dl_ok(A.ltab, A.max_dl, D.L, I.lo, I.lo + 3)) pc = 0;
                if (pc < 0) {
                    const int k = __ldg(A.order + kq);
                    int qp[3], qm[3];
                    pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + k), __ldg(A.grid.s64 + hq),
                                 __ldg(A.grid.c64 + hq), A.qkey, qp, qm);
                    if (CLIP) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            qp[c] = min(max(qp[c], 0), 255);
                            qm[c] = min(max(qm[c], 0), 255);
                        }
                    }
                    Decide dc{A.hi_min, A.lo_max, A.mask2, CLIP ? 1 : 0};
                    pc = decide_codes(qp, qm, dc);
                    if (pc > 0 && A.ltab && !dl_ok(A.ltab, A.max_dl, D.L, qp, qm)) pc = 0;
                    ++n_re;
                }
                if (pc > 0)
                    atomicMin(A.key + t * 7 + (pc - 1), ((uint32_t)kq << 16) | (uint32_t)hq);
            }
        }
    }
}

// One work item: target t, ranks [kk0, kk1) of the sorted radii.
template <int PREC, bool FAST, bool CLIP>
__device__ __forceinline__ void first_item(const FirstHitArgs& A, const float2* r2s,
                                           const float4* sc4s, const uint8_t* lut,
                                           const TargetF32& T, const ChainF32& C,
                                           const PairsC& PC, int64_t t, int kk0, int kk1,
                                           uint32_t* fb, unsigned long long& n_exact,
                                           unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    const int nslots = (kk1 - kk0) * H;
    const TargetF64 D = A.td[t];
    const PairsT P = make_pairs(T);
    uint32_t best[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) best[q] = kNoChoice;
    uint32_t found = 0;  // bit q: pattern q has an unflagged hit in this item
    const int q32 = 32 / H, r32 = 32 - q32 * H;
    int kk = kk0 + (int)lane / H, h = (int)lane % H;
    const int nit = (nslots + 31) >> 5;
    int it_pow = 0;  // iterations whose radii never reach the sRGB linear segment
    int it0 = 0;     // iterations wholly below the first radius where a pair may pass
    if (PREC == CVS_PREC_FP32_RECHECK && FAST) {
        const int ks = first_linseg_radius(T, C, r2s, kk0, kk1);
        it_pow = ks == kk1 ? nit : ((ks - kk0) * H) >> 5;
        const int kp = first_possible_radius(T, C, r2s, kk0, kk1, A.hi_min);
        if (kp > kk0) {
            it0 = kp == kk1 ? nit : ((kp - kk0) * H) >> 5;
            const int i = it0 * 32 + (int)lane;
            const int dk = i / H;
            kk = kk0 + dk;
            h = i - dk * H;
        }
    }
    for (int seg0 = it0; seg0 < nit; seg0 += kHitSegIters) {
        const int seg1 = min(seg0 + kHitSegIters, nit);
        for (int w = 0, it = seg0; it < seg1; ++w) {
            uint32_t bits = 0;
            const int wend = min(seg1, it + 32);
            for (uint32_t bit = 1u; it < wend; ++it, bit <<= 1) {
                const bool active = it * 32 + (int)lane < nslots;
                const int kq = active ? kk : kk0, hq = active ? h : 0;
                int pattern = 0;
                if (PREC == CVS_PREC_FP32_RECHECK) {
                    const float2 r2 = r2s[kq];
                    const float4 sc = sc4s[hq];
                    const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y));
                    const float2 w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
                    float2 lin[3];
                    lin32<FAST>(P, PC, u2, w2, lin);
                    // gamut reject: a warp whose pairs all leave the gamut has no hit
                    const bool skip = !CLIP && __all_sync(0xFFFFFFFFu, !active || surely_out32(lin));
                    if (!skip) {
                        int yp[3], ym[3];
                        bool flag;
                        if (it < it_pow) flag = encode32<false>(lin, A.half_w, yp, ym, nullptr);
                        else flag = encode32<true>(lin, A.half_w, yp, ym, nullptr);
                        pattern = decide32<CLIP>(yp, ym, lut, A.mask2);
                        flag = flag && active;
                        if (flag || !active) pattern = 0;
                        if (flag) bits |= bit;
                        if (pattern && A.ltab) {  // the luminance limit on the exact codes
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
                            if (!dl_ok(A.ltab, A.max_dl, D.L, qp, qm)) pattern = 0;
                        }
                    }
                } else if (active) {
                    const int k = __ldg(A.order + kq);
                    int qp[3], qm[3];
                    pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + k), __ldg(A.grid.s64 + hq),
                                 __ldg(A.grid.c64 + hq), A.qkey, qp, qm);
                    if (CLIP) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            qp[c] = min(max(qp[c], 0), 255);
                            qm[c] = min(max(qm[c], 0), 255);
                        }
                    }
                    Decide dc{A.hi_min, A.lo_max, A.mask2, CLIP ? 1 : 0};
                    pattern = decide_codes(qp, qm, dc);
                    if (pattern && A.ltab && !dl_ok(A.ltab, A.max_dl, D.L, qp, qm)) pattern = 0;
                }
                const uint32_t newp =
                    __reduce_or_sync(0xFFFFFFFFu, pattern ? (1u << pattern) : 0u) & ~found;
                if (newp) {  // the lowest lane holds the iteration's smallest key
                    const uint32_t mykey = ((uint32_t)kq << 16) | (uint32_t)hq;
#pragma unroll
                    for (int q = 1; q <= 7; ++q) {
                        if ((newp >> q) & 1u) {
                            const unsigned b = __ballot_sync(0xFFFFFFFFu, pattern == q);
                            best[q] = __shfl_sync(0xFFFFFFFFu, mykey, __ffs(b) - 1);
                        }
                    }
                    found |= newp;
                }
                h += r32;
                kk += q32;
                const bool wrap = h >= H;
                h = wrap ? h - H : h;
                kk = wrap ? kk + 1 : kk;
            }
            if (PREC == CVS_PREC_FP32_RECHECK) fb[w * 32 + lane] = bits;
        }
        if (PREC == CVS_PREC_FP32_RECHECK) {
            __syncwarp();
            first_flagged<PREC, FAST, CLIP>(A, r2s, sc4s, T, C, D, t, kk0, seg0,
                                            (seg1 - seg0 + 31) >> 5, fb, n_exact, n_re);
        }
    }
    uint32_t mine = kNoChoice;  // lane q - 1 publishes pattern q
#pragma unroll
    for (int q = 1; q <= 7; ++q)
        if ((int)lane == q - 1) mine = best[q];
    if ((int)lane < 7 && ((found >> (lane + 1)) & 1u)) atomicMin(A.key + t * 7 + lane, mine);
}

template <int PREC, bool CLIP>
__global__ void __launch_bounds__(kSearchBlock) k_first_hits(const FirstHitArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H;
    float2* r2s = reinterpret_cast<float2*>(smem);  // radii in rank order
    float4* sc4s = reinterpret_cast<float4*>(smem + ((K * 8 + 15) & ~15));
    uint8_t* lut = smem + ((K * 8 + 15) & ~15) + H * 16;
    uint32_t* fb = reinterpret_cast<uint32_t*>(lut + 3 * 512) + (threadIdx.x >> 5) * (kHitWords * 32);
    build_decide_lut(lut, A.hi_min, A.lo_max);
    for (int i = threadIdx.x; i < K; i += blockDim.x) r2s[i] = dup(A.grid.r32[A.order[i]]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        const float2 sc = A.grid.sc32[i];
        sc4s[i] = make_float4(sc.x, -sc.x, sc.y, -sc.y);
    }
    const unsigned lane = lane_id();
    for (int w = 0; w < kHitWords; ++w) fb[w * 32 + lane] = 0u;
    __syncthreads();
    ChainF32 C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C.Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        C.Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    const PairsC PC = make_pairs(C);
    unsigned long long n_exact = 0, n_re = 0;
    const int kchunk = A.kchunk;
    const int n_kc = (K + kchunk - 1) / kchunk;
    const unsigned long long n_items = (unsigned long long)A.n_targets * n_kc;
    while (true) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(A.work_counter, 1ull);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= n_items) break;
        const int64_t t = (int64_t)(item / (unsigned long long)n_kc);
        const int kc = (int)(item - (unsigned long long)t * n_kc);
        const int kk0 = kc * kchunk, kk1 = min(kk0 + kchunk, K);
        TargetF32 T{};
        if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
        if (PREC == CVS_PREC_FP32_RECHECK && (T.flags & 1u))
            first_item<PREC, true, CLIP>(A, r2s, sc4s, lut, T, C, PC, t, kk0, kk1, fb, n_exact,
                                         n_re);
        else
            first_item<PREC, false, CLIP>(A, r2s, sc4s, lut, T, C, PC, t, kk0, kk1, fb, n_exact,
                                          n_re);
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

// Keys -> table entries of 16 bytes (one sector read per lookup):
//   x = plus R | plus G << 8 | plus B << 16 | minus R << 24,
//   y = minus G | minus B << 8,  z = choice k | m << 16 (0xFFFFFFFF: none),  w = 0.
template <int PREC, bool CLIP>
__global__ void k_first_finalize(const FirstHitArgs A, const uint32_t* __restrict__ keys,
                                 uint4* __restrict__ entry) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.n_targets * 7) return;
    const uint32_t key = keys[e];
    if (key == kNoChoice) {
        entry[e] = make_uint4(0u, 0u, kNoChoice, 0u);
        return;
    }
    const int64_t t = e / 7;
    const int kk = (int)(key >> 16), h = (int)(key & 0xFFFFu);
    const int k = __ldg(A.order + kk);
    int qp[3], qm[3];
    bool exact = false;
    if (PREC == CVS_PREC_FP32_RECHECK) {
        const TargetF32 T = A.tf[t];
        ChainF32 C;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C.Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
            C.Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
        }
        const PairsT P = make_pairs(T);
        const PairsC PC = make_pairs(C);
        const float2 r2 = dup(A.grid.r32[k]);
        const float2 sc = A.grid.sc32[h];
        int yp[3], ym[3];
        bool flag;
        if (T.flags & 1u)
            flag = codes32<true, true>(P, PC, __fmul2_rn(r2, f2(sc.x, -sc.x)),
                                       __fmul2_rn(r2, f2(sc.y, -sc.y)), A.half_w, yp, ym);
        else
            flag = codes32<false, true>(P, PC, __fmul2_rn(r2, f2(sc.x, -sc.x)),
                                        __fmul2_rn(r2, f2(sc.y, -sc.y)), A.half_w, yp, ym);
        if (!flag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                qp[c] = yp[c] - kMagicBits;
                qm[c] = ym[c] - kMagicBits;
            }
            exact = true;
        }
    }
    if (!exact) {
        const TargetF64 D = A.td[t];
        pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + k), __ldg(A.grid.s64 + h),
                     __ldg(A.grid.c64 + h), A.qkey, qp, qm);
    }
    uint64_t v = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a = CLIP ? min(max(qp[c], 0), 255) : qp[c];
        const int b = CLIP ? min(max(qm[c], 0), 255) : qm[c];
        v |= (uint64_t)(uint8_t)a << (8 * c);
        v |= (uint64_t)(uint8_t)b << (8 * (3 + c));
    }
    entry[e] = make_uint4((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)k | ((uint32_t)h << 16), 0u);
}

// Frames of one image from the table: grid-stride over pixels, four pixels per
// thread per step so that four table reads are in flight at once.
__global__ void k_etab_gather(const uint4* __restrict__ entry, const uint8_t* __restrict__ rgb,
                              int64_t pitch, int32_t width, int64_t n,
                              const uint8_t* __restrict__ pattern, int64_t pattern_pitch,
                              uint8_t* __restrict__ frame_a, uint8_t* __restrict__ frame_b,
                              int64_t frame_pitch, uint32_t* __restrict__ choice_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n;
         base += 4 * stride) {
        uint32_t src[4];
        uint4 e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = base + u * stride;
            e[u] = make_uint4(0u, 0u, kNoChoice, 0u);
            src[u] = 0;
            if (t < n) {
                const int64_t y = t / width, x = t - y * width;
                const uint8_t* px = rgb + y * pitch + 3 * x;
                src[u] = (uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16);
                const int p = pattern[y * pattern_pitch + x];
                if (p >= 1 && p <= 7) {
                    const int64_t c = ((int64_t)px[0] << 16) | ((int64_t)px[1] << 8) | px[2];
                    e[u] = __ldg(entry + c * 7 + (p - 1));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = base + u * stride;
            if (t >= n) continue;
            const int64_t y = t / width, x = t - y * width;
            uint8_t* fa = frame_a + y * frame_pitch + 3 * x;
            uint8_t* fb = frame_b + y * frame_pitch + 3 * x;
            const bool hit = e[u].z != kNoChoice;
            const uint32_t a = hit ? e[u].x : src[u];
            const uint32_t b = hit ? ((e[u].x >> 24) | (e[u].y << 8)) : src[u];
            fa[0] = (uint8_t)a; fa[1] = (uint8_t)(a >> 8); fa[2] = (uint8_t)(a >> 16);
            fb[0] = (uint8_t)b; fb[1] = (uint8_t)(b >> 8); fb[2] = (uint8_t)(b >> 16);
            if (choice_out) choice_out[t] = e[u].z;
        }
    }
}

int embed_smem_bytes(const GridDev& g) { return ((g.K * 8 + 15) & ~15) + g.H * 16 + 3 * 512; }

int first_smem_bytes(const GridDev& g) {
    return embed_smem_bytes(g) + (kSearchBlock / 32) * kHitWords * 32 * 4;
}

template <int PREC, bool CLIP>
cudaError_t launch_first_t(const FirstHitArgs& a, cudaStream_t st) {
    const int smem = first_smem_bytes(a.grid);
    const void* fn = (const void*)k_first_hits<PREC, CLIP>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSearchBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_first_hits<PREC, CLIP><<<a.num_sms * per_sm, kSearchBlock, smem, st>>>(a);
    return cudaGetLastError();
}

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

cudaError_t launch_first_hits(const FirstHitArgs& a, cudaStream_t st) {
    if (a.n_targets <= 0) return cudaSuccess;
    if (a.prec == CVS_PREC_FP64)
        return a.clip ? launch_first_t<CVS_PREC_FP64, true>(a, st)
                      : launch_first_t<CVS_PREC_FP64, false>(a, st);
    return a.clip ? launch_first_t<CVS_PREC_FP32_RECHECK, true>(a, st)
                  : launch_first_t<CVS_PREC_FP32_RECHECK, false>(a, st);
}

cudaError_t launch_first_finalize(const FirstHitArgs& a, const uint32_t* keys, uint4* entry,
                                  cudaStream_t st) {
    const int64_t n = a.n_targets * 7;
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256);
    if (a.prec == CVS_PREC_FP64) {
        if (a.clip) k_first_finalize<CVS_PREC_FP64, true><<<blocks, 256, 0, st>>>(a, keys, entry);
        else k_first_finalize<CVS_PREC_FP64, false><<<blocks, 256, 0, st>>>(a, keys, entry);
    } else {
        if (a.clip)
            k_first_finalize<CVS_PREC_FP32_RECHECK, true><<<blocks, 256, 0, st>>>(a, keys, entry);
        else
            k_first_finalize<CVS_PREC_FP32_RECHECK, false><<<blocks, 256, 0, st>>>(a, keys, entry);
    }
    return cudaGetLastError();
}

cudaError_t launch_etab_gather(const uint4* entry, const uint8_t* rgb, int64_t pitch,
                               int32_t width, int32_t height, const uint8_t* pattern,
                               int64_t pattern_pitch, uint8_t* frame_a, uint8_t* frame_b,
                               int64_t frame_pitch, uint32_t* choice_out, cudaStream_t st) {
    const int64_t n = (int64_t)width * height;
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 1023) / 1024, cap = (int64_t)(sms > 0 ? sms : 1) * 16;
    k_etab_gather<<<(int)(want < cap ? want : cap), 256, 0, st>>>(
        entry, rgb, pitch, width, n, pattern, pattern_pitch, frame_a, frame_b, frame_pitch,
        choice_out);
    return cudaGetLastError();
}

cudaError_t launch_embed(const EmbedArgs& a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    if (a.prec == CVS_PREC_FP64)
        return a.clip ? launch_embed_t<CVS_PREC_FP64, true>(a, st)
                      : launch_embed_t<CVS_PREC_FP64, false>(a, st);
    return a.clip ? launch_embed_t<CVS_PREC_FP32_RECHECK, true>(a, st)
                  : launch_embed_t<CVS_PREC_FP32_RECHECK, false>(a, st);
}

}  // namespace cvs
