// cvs_multi.cu - the multi-threshold colour-pair search (sm_103a): every
// candidate decided against up to kMaxThresholdSets (V_th, R_novib, mask) sets
// in one pass (§3 Experiments, Table 1).
#include <cuda_runtime.h>

#include "cvs_device.cuh"
#include "cvs_internal.h"
#include "cvs_slot32.cuh"

namespace cvs {

namespace {

// ------------------------------------------------------------ multi-threshold search
// The paper's experiment (§3 Experiments, Table 1): every candidate decided
// against n_thr threshold sets in one pass.  The pair chain runs once per slot;
// each set has its own classification table; per set the warp's passes are
// reduced with ballot / REDUX and lane s keeps set s's running totals.
template <int PREC, bool FAST, bool CLIP>
__device__ __forceinline__ void multi_item(const MultiArgs& A, const float2* r2s, const float4* sc4s,
                                           const uint8_t* luts, int64_t t, int k0, int k1,
                                           const ChainF32& C, uint32_t* pq, uint32_t* rq_kh,
                                           unsigned long long& n_flag, unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H, NT = A.n_thr;
    const int inc = A.grid.sym ? 2 : 1;
    const int nslots = (k1 - k0) * H;
    TargetF32 T;
    TargetF64 D;
    if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
    else D = A.td[t];
    const PairsT P = make_pairs(T);
    const PairsC PC = make_pairs(C);
    int cnt = 0;
    uint32_t rbits = 0, pm = 0;  // set `lane`'s totals (lanes < NT)
    int pq_n = 0;
    // one warp-wide merge of per-lane patterns of set s into lane s's totals
    auto merge = [&](int s, int pattern, float r) {
        const bool pass = pattern > 0;
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, pass);
        if (ball) {
            const uint32_t pmw = __reduce_or_sync(0xFFFFFFFFu, pass ? (1u << pattern) : 0u);
            const uint32_t rmw = __reduce_max_sync(0xFFFFFFFFu, pass ? __float_as_uint(r) : 0u);
            if ((int)lane == s) {
                cnt += __popc(ball) * inc;
                pm |= pmw;
                rbits = max(rbits, rmw);
            }
        }
    };
    // flagged slots: bounds once, then every set; FP64 when some set is undecided
    auto drain = [&](int n) {
        int k = 0, h = 0;
        Intervals I{};
        float r = 0.0f;
        const bool mine = (int)lane < n;
        if (mine) {
            const uint32_t kh = pq[lane];
            k = (int)(kh & 0xFFFFu);
            h = (int)(kh >> 16);
            r = r2s[k].x;
            const float4 sc = sc4s[h];
            I = intervals32<FAST>(T, C, r2s[k], sc, A.half_w, CLIP ? 1 : 0);
        }
        bool need64 = false;
        for (int s = 0; s < NT; ++s) {
            const int pc = mine ? certain_from(I, A.hi_min[s], A.lo_max[s], A.mask2[s], CLIP ? 1 : 0, 0)
                                : 0;
            need64 |= pc < 0;
            merge(s, pc < 0 ? 0 : pc, r);
        }
        // slots with an undecided set: exact FP64 codes, every set decided from them
        // (the sets decided above are decided again identically, so count only here)
        const unsigned b64 = __ballot_sync(0xFFFFFFFFu, need64);
        if (b64) {
            int qp[3] = {0, 0, 0}, qm[3] = {0, 0, 0};
            if (need64) {
                const double rr = __ldg(A.grid.r64 + k), ss = __ldg(A.grid.s64 + h),
                             cc = __ldg(A.grid.c64 + h);
                const TargetF64 DD = A.td[t];
                pair_codes64(DD.L, DD.a, DD.b, rr, ss, cc, A.qkey, qp, qm);
                if (CLIP) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        qp[i] = min(max(qp[i], 0), 255);
                        qm[i] = min(max(qm[i], 0), 255);
                    }
                }
                ++n_re;
            }
            for (int s = 0; s < NT; ++s) {
                int pat = 0;
                if (need64) {
                    const int pc = certain_from(I, A.hi_min[s], A.lo_max[s], A.mask2[s],
                                                CLIP ? 1 : 0, 0);
                    if (pc < 0) {  // undecided in FP32: the FP64 decision counts now
                        Decide dc{A.hi_min[s], A.lo_max[s], A.mask2[s], CLIP ? 1 : 0};
                        pat = decide_codes(qp, qm, dc);
                    }
                }
                merge(s, pat, r);
            }
        }
        __syncwarp();
    };
    const int q32 = 32 / H, r32 = 32 - q32 * H;
    int k = k0 + (int)lane / H, h = (int)lane % H;
    const int nit = (nslots + 31) >> 5;
    int it_pow = 0;  // iterations whose radii never reach the sRGB linear segment
    int it0 = 0;     // iterations wholly below the first radius where some set may pass
    if (PREC == CVS_PREC_FP32_RECHECK && FAST) {
        const int k_split = first_linseg_radius(T, C, r2s, k0, k1);
        it_pow = k_split == k1 ? nit : ((k_split - k0) * H) >> 5;
        const int kp = first_possible_radius(T, C, r2s, k0, k1, A.hi_min_all);
        if (kp > k0) {
            it0 = kp == k1 ? nit : ((kp - k0) * H) >> 5;
            const int i = it0 * 32 + (int)lane;
            const int dk = i / H;
            k = k0 + dk;
            h = i - dk * H;
        }
    }
    for (int it = it0; it < nit; ++it) {
        const bool active = it * 32 + (int)lane < nslots;
        const int kk = active ? k : k0, hh = active ? h : 0;
        const float2 r2 = r2s[kk];
        int yp[3], ym[3], qp[3], qm[3];
        bool flag = false;
        if (PREC == CVS_PREC_FP32_RECHECK) {
            const float4 sc = sc4s[hh];
            const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y)), w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
            float2 lin[3];
            lin32<FAST>(P, PC, u2, w2, lin);
            // gamut reject: a warp whose pairs all leave the gamut passes no set
            if (!CLIP && __all_sync(0xFFFFFFFFu, !active || surely_out32(lin))) {
                h += r32;
                k += q32;
                const bool wrap = h >= H;
                h = wrap ? h - H : h;
                k = wrap ? k + 1 : k;
                continue;
            }
            if (it < it_pow) flag = encode32<false>(lin, A.half_w, yp, ym, nullptr);
            else flag = encode32<true>(lin, A.half_w, yp, ym, nullptr);
            flag = flag && active;
        } else if (active) {
            pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + kk), __ldg(A.grid.s64 + hh),
                         __ldg(A.grid.c64 + hh), A.qkey, qp, qm);
            if (CLIP) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    qp[i] = min(max(qp[i], 0), 255);
                    qm[i] = min(max(qm[i], 0), 255);
                }
            }
        }
        for (int s = 0; s < NT; ++s) {
            int pattern = 0;
            if (PREC == CVS_PREC_FP32_RECHECK) {
                pattern = decide32<CLIP>(yp, ym, luts + s * 3 * 512, A.mask2[s]);
                if (flag || !active) pattern = 0;
            } else if (active) {
                Decide dc{A.hi_min[s], A.lo_max[s], A.mask2[s], CLIP ? 1 : 0};
                pattern = decide_codes(qp, qm, dc);
            }
            merge(s, pattern, r2.x);
        }
        if (PREC == CVS_PREC_FP32_RECHECK) {
            const unsigned fball = __ballot_sync(0xFFFFFFFFu, flag);
            if (fball) {
                if (flag) {
                    pq[pq_n + __popc(fball & ((1u << lane) - 1u))] = (uint32_t)kk | ((uint32_t)hh << 16);
                    ++n_flag;
                }
                pq_n += __popc(fball);
                __syncwarp();
                if (pq_n >= 32) {
                    drain(32);
                    const int rest = pq_n - 32;
                    const uint32_t mv = (int)lane < rest ? pq[32 + lane] : 0u;
                    __syncwarp();
                    if ((int)lane < rest) pq[lane] = mv;
                    __syncwarp();
                    pq_n = rest;
                }
            }
        }
        h += r32;
        k += q32;
        const bool wrap = h >= H;
        h = wrap ? h - H : h;
        k = wrap ? k + 1 : k;
    }
    if (PREC == CVS_PREC_FP32_RECHECK && pq_n > 0) drain(pq_n);
    if ((int)lane < NT && cnt) {
        Acc* ac = A.acc + t * NT + lane;
        atomicAdd(&ac->count, cnt);
        atomicMax(&ac->rmax_bits, (int)rbits);
        atomicOr(&ac->pmask, pm >> 1);
    }
    (void)rq_kh;
}

template <int PREC, bool CLIP>
__global__ void __launch_bounds__(kSearchBlock) k_search_multi(const MultiArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H, NT = A.n_thr;
    float2* r2s = reinterpret_cast<float2*>(smem);
    float4* sc4s = reinterpret_cast<float4*>(smem + ((K * 8 + 15) & ~15));
    uint8_t* luts = smem + ((K * 8 + 15) & ~15) + H * 16;
    uint32_t* pq_all = reinterpret_cast<uint32_t*>(luts + ((NT * 3 * 512 + 15) & ~15));
    const int warp = threadIdx.x >> 5;
    uint32_t* pq = pq_all + warp * kRqCap;
    for (int s2 = 0; s2 < NT; ++s2) build_decide_lut(luts + s2 * 3 * 512, A.hi_min[s2], A.lo_max[s2]);
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
    unsigned long long n_flag = 0, n_re = 0;
    const int kchunk = A.kchunk;
    const int n_kc = (K + kchunk - 1) / kchunk;
    const unsigned long long n_items = (unsigned long long)A.n_targets * n_kc;
    const unsigned lane = lane_id();
    while (true) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(A.work_counter, 1ull);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= n_items) break;
        const int64_t t = (int64_t)(item / (unsigned long long)n_kc);
        const int kc = (int)(item - (unsigned long long)t * n_kc);
        const int k0 = kc * kchunk, k1 = min(k0 + kchunk, K);
        if (PREC == CVS_PREC_FP32_RECHECK) {
            if (A.tf[t].flags & 1u)
                multi_item<PREC, true, CLIP>(A, r2s, sc4s, luts, t, k0, k1, C, pq, nullptr, n_flag, n_re);
            else
                multi_item<PREC, false, CLIP>(A, r2s, sc4s, luts, t, k0, k1, C, pq, nullptr, n_flag, n_re);
        } else {
            multi_item<PREC, true, CLIP>(A, r2s, sc4s, luts, t, k0, k1, C, pq, nullptr, n_flag, n_re);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n_flag += __shfl_xor_sync(0xFFFFFFFFu, n_flag, off);
        n_re += __shfl_xor_sync(0xFFFFFFFFu, n_re, off);
    }
    if (lane == 0) {
        if (n_flag) atomicAdd(A.stats + 0, n_flag);
        if (n_re) atomicAdd(A.stats + 1, n_re);
    }
}

__global__ void k_init_acc(Acc* __restrict__ acc, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Acc z;
    z.count = 0;
    z.rmax_bits = __float_as_int(-1.0f);
    z.pmask = 0;
    z.pad = 0;
    acc[i] = z;
}

}  // namespace

int multi_smem_bytes(const GridDev& g, int n_thr, int block) {
    return ((g.K * 8 + 15) & ~15) + g.H * 16 + ((n_thr * 3 * 512 + 15) & ~15) +
           (block / 32) * kRqCap * 4;
}

template <int PREC, bool CLIP>
cudaError_t launch_multi_t(const MultiArgs& a, int block, cudaStream_t st) {
    const int smem = multi_smem_bytes(a.grid, a.n_thr, block);
    const void* fn = (const void*)k_search_multi<PREC, CLIP>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_search_multi<PREC, CLIP><<<a.num_sms * per_sm, block, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_search_multi(const MultiArgs& a, cudaStream_t st) {
    const int block = kSearchBlock;
    if (a.prec == CVS_PREC_FP64)
        return a.clip ? launch_multi_t<CVS_PREC_FP64, true>(a, block, st)
                      : launch_multi_t<CVS_PREC_FP64, false>(a, block, st);
    return a.clip ? launch_multi_t<CVS_PREC_FP32_RECHECK, true>(a, block, st)
                  : launch_multi_t<CVS_PREC_FP32_RECHECK, false>(a, block, st);
}

cudaError_t launch_init_acc(Acc* acc, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_init_acc<<<(int)((n + 255) / 256), 256, 0, st>>>(acc, n);
    return cudaGetLastError();
}

}  // namespace cvs
