// cvs_kernels.cu - CUDA kernels of libcvsearch (sm_103a).
//
// Hot path (paper §2 Methods, §3 Experiments, Table 1), per target colour:
//   setup   : 8-bit sRGB -> L*a*b* in FP64 (correctly rounded cube roots), and
//             the FP32 constants of the relative inverse chain (one thread each)
//   search  : persistent warps pull (target, radius chunk) items from an atomic
//             work counter; lanes stride over (radius k, angle slot h); each
//             slot forms the point-symmetric pair (a +- D_a, b +- D_b) at fixed
//             L*, converts both colours to 8-bit sRGB in FP32 (FMA + MUFU),
//             tests gamut and the V_th / R_novib embedding-signal condition,
//             and reduces count / max radius / pattern mask per warp.  Slots
//             whose FP32 codes sit within W of a rounding boundary, and whose
//             decision could change, are queued in shared memory and
//             re-decided 32 at a time in FP64 (one slot per lane).
//   finalize: per-target accumulators -> caller's capacity maps.
// When the angle list is closed under +180 degrees, slot h covers angles h and
// h + N/2: the "minus" colour of one is the "plus" colour of the other.
#include <cuda_runtime.h>

#include "cvs_device.cuh"
#include "cvs_internal.h"

namespace cvs {

namespace {

constexpr int kRqCap = 64;  // re-decision queue entries per warp

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// ------------------------------------------------------------ trig table
__global__ void k_trig_table(const double* __restrict__ ang, int n, double* s64, double* c64,
                             float2* sc32, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s, c;
    int unc = 0;
    sincos_deg_rn(ang[i], &s, &c, &unc);
    s64[i] = s;
    c64[i] = c;
    sc32[i] = make_float2(__double2float_rn(__ddiv_rn(s, 500.0)),
                          __double2float_rn(__ddiv_rn(-c, 200.0)) + 0.0f);
    if (unc) atomicOr(status, 1);
}

// ------------------------------------------------------------ target setup
__device__ __forceinline__ void setup_one(uint32_t r8, uint32_t g8, uint32_t b8, double rmax,
                                          uint64_t slot, TargetF32* __restrict__ tf,
                                          TargetF64* __restrict__ td, Acc* __restrict__ acc,
                                          int64_t t) {
    double L, a, b;
    target_lab64(r8, g8, b8, L, a, b);
    // The FP64 inverse chain at radius 0, operation for operation.
    const double fy = __ddiv_rn(__dadd_rn(L, 16.0), 116.0);
    const double fx0 = __dadd_rn(fy, __ddiv_rn(a, 500.0));
    const double fz0 = __dsub_rn(fy, __ddiv_rn(b, 200.0));
    const double X3 = cie_finv64(fx0), Y3 = cie_finv64(fy), Z3 = cie_finv64(fz0);
    const double X = __dmul_rn(c_W[0], X3), Y = __dmul_rn(c_W[1], Y3), Z = __dmul_rn(c_W[2], Z3);
    TargetF32 o;
    o.c1x = __double2float_rn(3.0 * fx0);
    o.c2x = __double2float_rn(3.0 * fx0 * fx0);
    o.c1z = __double2float_rn(3.0 * fz0);
    o.c2z = __double2float_rn(3.0 * fz0 * fz0);
    o.fx0 = __double2float_rn(fx0);
    o.fz0 = __double2float_rn(fz0);
    o.X30 = __double2float_rn(X3);
    o.Z30 = __double2float_rn(Z3);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double lin = __dadd_rn(__dadd_rn(__dmul_rn(c_MI[3 * c], X), __dmul_rn(c_MI[3 * c + 1], Y)),
                                     __dmul_rn(c_MI[3 * c + 2], Z));
        o.lin0[c] = __double2float_rn(lin);
    }
    // Fast path: every candidate's f-values stay above 6/29 (cubic branch).
    const double umax = rmax / 500.0 * (1.0 + 1e-9), wmax = rmax / 200.0 * (1.0 + 1e-9);
    const double lim = kFinvBreak * (1.0 + 1e-9);
    o.flags = (fx0 - umax > lim && fz0 - wmax > lim) ? 1u : 0u;
    tf[t] = o;
    TargetF64 d;
    d.L = L;
    d.a = a;
    d.b = b;
    d.out_slot = slot;
    td[t] = d;
    Acc z;
    z.count = 0;
    z.rmax_bits = __float_as_int(-1.0f);
    z.pmask = 0;
    z.pad = 0;
    acc[t] = z;
}

__global__ void k_setup_colors(const uint8_t* __restrict__ rgb, int64_t n, double rmax,
                               TargetF32* tf, TargetF64* td, Acc* acc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    setup_one(rgb[3 * t], rgb[3 * t + 1], rgb[3 * t + 2], rmax, (uint64_t)t, tf, td, acc, t);
}

__device__ __forceinline__ int find_image(const ImageDesc* imgs, int n_imgs, int64_t p) {
    int lo = 0, hi = n_imgs - 1;  // largest i with imgs[i].first <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].first <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_setup_images(const ImageDesc* __restrict__ imgs, int n_imgs, int64_t total,
                               double rmax, TargetF32* tf, TargetF64* td, Acc* acc) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int i = find_image(imgs, n_imgs, p);
    const ImageDesc im = imgs[i];
    const int64_t local = p - im.first;
    const int64_t y = local / im.width, x = local - y * im.width;
    const uint8_t* px = im.rgb + y * im.pitch + 3 * x;
    setup_one(px[0], px[1], px[2], rmax, ((uint64_t)i << 40) | (uint64_t)local, tf, td, acc, p);
}

// ------------------------------------------------------------ FP32 slot
// Codes of the pair at displacement (u, w) = (r sin j / 500, -r cos j / 200) in
// f-space, as biased integers y = kMagicBits + q.  Returns true if some code's
// unrounded value lies within W of a rounding boundary.
template <bool FAST>
__device__ __forceinline__ bool codes32(const TargetF32& T, const float Ax[3], const float Bz[3],
                                        float u, float w, float half_w, int yp[3], int ym[3]) {
    float dXp, dXm, dZp, dZm;
    if (FAST) {
        dXp = u * fmaf(u, T.c1x + u, T.c2x);
        dXm = -u * fmaf(-u, T.c1x - u, T.c2x);
        dZp = w * fmaf(w, T.c1z + w, T.c2z);
        dZm = -w * fmaf(-w, T.c1z - w, T.c2z);
    } else {
        const float brk = (float)kFinvBreak, add = (float)kFLinAdd, mul = (float)kFinvLinMul;
        const float fxp = T.fx0 + u, fxm = T.fx0 - u, fzp = T.fz0 + w, fzm = T.fz0 - w;
        dXp = (fxp > brk ? fxp * fxp * fxp : (fxp - add) * mul) - T.X30;
        dXm = (fxm > brk ? fxm * fxm * fxm : (fxm - add) * mul) - T.X30;
        dZp = (fzp > brk ? fzp * fzp * fzp : (fzp - add) * mul) - T.Z30;
        dZm = (fzm > brk ? fzm * fzm * fzm : (fzm - add) * mul) - T.Z30;
    }
    bool flag = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float lp = fmaf(Bz[c], dZp, fmaf(Ax[c], dXp, T.lin0[c]));
        const float lm = fmaf(Bz[c], dZm, fmaf(Ax[c], dXm, T.lin0[c]));
        const float vp = encode_v32(lp), vm = encode_v32(lm);
        const float yfp = __fadd_rn(vp, kMagic), yfm = __fadd_rn(vm, kMagic);
        flag |= fabsf(__fsub_rn(vp, __fsub_rn(yfp, kMagic))) >= half_w;
        flag |= fabsf(__fsub_rn(vm, __fsub_rn(yfm, kMagic))) >= half_w;
        yp[c] = __float_as_int(yfp);
        ym[c] = __float_as_int(yfm);
    }
    return flag;
}

// Embedding-signal decision on biased codes (exact when no code is flagged).
__device__ __forceinline__ int decide32(const int yp_in[3], const int ym_in[3], int32_t hi_min,
                                        int32_t lo_max, uint32_t mask2, int32_t clip) {
    int yp[3], ym[3];
    uint32_t out = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        yp[c] = yp_in[c];
        ym[c] = ym_in[c];
        if (clip) {
            yp[c] = min(max(yp[c], kMagicBits), kMagicBits + 255);
            ym[c] = min(max(ym[c], kMagicBits), kMagicBits + 255);
        }
        out |= ((uint32_t)yp[c] ^ (uint32_t)kMagicBits) | ((uint32_t)ym[c] ^ (uint32_t)kMagicBits);
    }
    const uint32_t gap = (uint32_t)(hi_min - lo_max - 1);
    bool invalid = out > 255u;  // a code outside [0, 255] (reject mode)
    uint32_t pattern = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int d = abs(yp[c] - ym[c]);
        invalid |= (uint32_t)(d - lo_max - 1) < gap;
        pattern |= ((uint32_t)(hi_min - 1 - d) >> 31) << (2 - c);
    }
    const bool ok = !invalid && ((mask2 >> pattern) & 1u);
    return ok ? (int)pattern : 0;
}

// Exact analysis of a slot with flagged codes: each flagged code may be one
// off towards its nearby boundary.  Returns 1 if the FP32 decision is certain
// (*pattern_out is then exact), 0 if an FP64 re-decision is needed.
// Return value: -1 = re-decide in FP64, else the exact pattern (0 = fail).
template <bool FAST>
__device__ __noinline__ int certain32(const TargetF32 T, const ChainF32 C, float u, float w,
                                      float half_w, int32_t hi_min, int32_t lo_max,
                                      uint32_t mask2, int32_t clip, int list_mode) {
    const float* Ax = C.Ax;
    const float* Bz = C.Bz;
    // recompute the unrounded values
    float dXp, dXm, dZp, dZm;
    if (FAST) {
        dXp = u * fmaf(u, T.c1x + u, T.c2x);
        dXm = -u * fmaf(-u, T.c1x - u, T.c2x);
        dZp = w * fmaf(w, T.c1z + w, T.c2z);
        dZm = -w * fmaf(-w, T.c1z - w, T.c2z);
    } else {
        const float brk = (float)kFinvBreak, add = (float)kFLinAdd, mul = (float)kFinvLinMul;
        const float fxp = T.fx0 + u, fxm = T.fx0 - u, fzp = T.fz0 + w, fzm = T.fz0 - w;
        dXp = (fxp > brk ? fxp * fxp * fxp : (fxp - add) * mul) - T.X30;
        dXm = (fxm > brk ? fxm * fxm * fxm : (fxm - add) * mul) - T.X30;
        dZp = (fzp > brk ? fzp * fzp * fzp : (fzp - add) * mul) - T.Z30;
        dZm = (fzm > brk ? fzm * fzm * fzm : (fzm - add) * mul) - T.Z30;
    }
    int lo[6], hi[6];  // code intervals: values 0..2 plus colour, 3..5 minus colour
    bool any_flag = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float dX = s ? dXm : dXp, dZ = s ? dZm : dZp;
            const float lin = fmaf(Bz[c], dZ, fmaf(Ax[c], dX, T.lin0[c]));
            const float v = encode_v32(lin);
            const float rr = __fsub_rn(__fadd_rn(v, kMagic), kMagic);
            const int q = (int)rr;
            const float d = __fsub_rn(v, rr);
            const bool f = fabsf(d) >= half_w;
            any_flag |= f;
            const int j = 3 * s + c;
            lo[j] = q - ((f && d < 0.0f) ? 1 : 0);
            hi[j] = q + ((f && d >= 0.0f) ? 1 : 0);
            if (clip) {
                lo[j] = min(max(lo[j], 0), 255);
                hi[j] = min(max(hi[j], 0), 255);
            }
        }
    }
    bool certain_out = false, maybe_out = false;
    if (!clip) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            certain_out |= hi[j] < 0 || lo[j] > 255;
            maybe_out |= lo[j] < 0 || hi[j] > 255;
        }
    }
    if (certain_out) return 0;
    bool certain_invalid = false, unstable = maybe_out;
    int pattern = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int dmax = max(hi[c] - lo[3 + c], hi[3 + c] - lo[c]);
        const int dmin = max(0, max(lo[c] - hi[3 + c], lo[3 + c] - hi[c]));
        const int cls_lo = dmin >= hi_min ? 2 : (dmin <= lo_max ? 0 : 1);
        const int cls_hi = dmax >= hi_min ? 2 : (dmax <= lo_max ? 0 : 1);
        if (cls_lo == 1 && cls_hi == 1) certain_invalid = true;
        if (cls_lo != cls_hi) unstable = true;
        pattern |= (cls_lo == 2 ? 1 : 0) << (2 - c);
    }
    if (certain_invalid) return 0;
    if (unstable) return -1;
    const bool ok = (mask2 >> pattern) & 1u;
    // a list needs the exact codes of a passing pair
    if (ok && list_mode && any_flag) return -1;
    return ok ? pattern : 0;
}

// ------------------------------------------------------------ search kernel
struct Smem {
    float* r;       // K
    float2* sc;     // H used
    uint32_t* rq_t; // per warp: kRqCap target indices (low 32 bits)
    uint32_t* rq_kh;
};

__device__ __forceinline__ void write_records(cvs_pair* dense, int N, int H, int sym, int k, int h,
                                              const int qp[3], const int qm[3], int pattern,
                                              uint32_t flags, uint32_t target) {
    cvs_pair rec;
    rec.k = (uint16_t)k;
    rec.m = (uint16_t)h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rec.plus[c] = (uint8_t)qp[c];
        rec.minus[c] = (uint8_t)qm[c];
    }
    rec.pattern = (uint8_t)pattern;
    rec.flags = (uint8_t)flags;
    rec.target = target;
    dense[(int64_t)k * N + h] = rec;
    if (sym) {
        rec.m = (uint16_t)(h + H);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rec.plus[c] = (uint8_t)qm[c];
            rec.minus[c] = (uint8_t)qp[c];
        }
        dense[(int64_t)k * N + h + H] = rec;
    }
}

// Exact FP64 decision of one slot; returns the pattern (0 = fail) and the
// emitted codes (clamped in clip mode).
__device__ __forceinline__ int decide64_slot(const SearchArgs& A, const TargetF64& D, int k, int h,
                                             int qp[3], int qm[3]) {
    const double r = __ldg(A.grid.r64 + k), s = __ldg(A.grid.s64 + h), c = __ldg(A.grid.c64 + h);
    pair_codes64(D.L, D.a, D.b, r, s, c, A.qkey, qp, qm);
    Decide dc;
    dc.hi_min = A.hi_min;
    dc.lo_max = A.lo_max;
    dc.mask2 = A.mask2;
    dc.clip = A.clip;
    if (A.clip) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            qp[i] = min(max(qp[i], 0), 255);
            qm[i] = min(max(qm[i], 0), 255);
        }
    }
    return decide_codes(qp, qm, dc);
}

// Re-decide up to 32 queued slots in FP64, one per lane, and merge them.
__device__ __noinline__ void flush_queue(const SearchArgs& A, uint32_t* rq_t, uint32_t* rq_kh,
                                         int n, unsigned long long* n_re) {
    const unsigned lane = lane_id();
    const int inc = A.grid.sym ? 2 : 1;
    if ((int)lane < n) {
        const uint32_t t = rq_t[lane];
        const uint32_t kh = rq_kh[lane];
        const int k = (int)(kh & 0xFFFFu), h = (int)(kh >> 16);
        const TargetF64 D = A.td[t];
        int qp[3], qm[3];
        const int pat = decide64_slot(A, D, k, h, qp, qm);
        if (pat) {
            if (A.list_mode) {
                write_records(A.dense, A.grid.N, A.grid.H, A.grid.sym, k, h, qp, qm, pat, 1u,
                              A.target_id);
            } else {
                Acc* ac = A.acc + t;
                atomicAdd(&ac->count, inc);
                atomicMax(&ac->rmax_bits, __float_as_int(__ldg(A.grid.r32 + k)));
                atomicOr(&ac->pmask, 1u << (pat - 1));
            }
        }
        *n_re += 1;
    }
    __syncwarp();
}

template <int PREC, bool FAST>
__device__ __forceinline__ void run_item(const SearchArgs& A, const Smem& S, int64_t t, int k0,
                                         int k1, const float Ax[3], const float Bz[3],
                                         uint32_t* rq_t, uint32_t* rq_kh, int& rq_n,
                                         unsigned long long& n_flag, unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    const int inc = A.grid.sym ? 2 : 1;
    const int nslots = (k1 - k0) * H;
    TargetF32 T;
    TargetF64 D;
    if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
    else D = A.td[t];
    int cnt = 0;
    float rmax = -1.0f;
    uint32_t pm = 0;
    // lane's first slot
    int k = k0 + (int)lane / H, h = (int)lane % H;
    for (int base = 0; base < nslots; base += 32) {
        const bool active = base + (int)lane < nslots;
        const int kk = active ? k : k0, hh = active ? h : 0;
        const float r = S.r[kk];
        int pattern = 0;
        bool need64 = false;
        int qp[3], qm[3];
        if (PREC == CVS_PREC_FP32_RECHECK) {
            const float2 sc = S.sc[hh];
            const float u = r * sc.x, w = r * sc.y;
            int yp[3], ym[3];
            const bool flag = codes32<FAST>(T, Ax, Bz, u, w, A.half_w, yp, ym) && active;
            pattern = decide32(yp, ym, A.hi_min, A.lo_max, A.mask2, A.clip);
            if (flag) {
                ++n_flag;
                ChainF32 C;
#pragma unroll
                for (int c = 0; c < 3; ++c) { C.Ax[c] = Ax[c]; C.Bz[c] = Bz[c]; }
                const int pc = certain32<FAST>(T, C, u, w, A.half_w, A.hi_min, A.lo_max, A.mask2,
                                               A.clip, A.list_mode);
                need64 = pc < 0;
                pattern = pc < 0 ? 0 : pc;
            }
            if (A.list_mode && pattern && active) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int a = yp[c] - kMagicBits, b = ym[c] - kMagicBits;
                    if (A.clip) { a = min(max(a, 0), 255); b = min(max(b, 0), 255); }
                    qp[c] = a;
                    qm[c] = b;
                }
            }
        } else {
            pattern = active ? decide64_slot(A, D, kk, hh, qp, qm) : 0;
        }
        if (!active) pattern = 0;
        if (pattern) {
            if (A.list_mode) {
                write_records(A.dense, A.grid.N, H, A.grid.sym, kk, hh, qp, qm, pattern, 0u,
                              A.target_id);
            } else {
                cnt += inc;
                rmax = fmaxf(rmax, r);
                pm |= 1u << (pattern - 1);
            }
        }
        if (PREC == CVS_PREC_FP32_RECHECK) {
            const unsigned ball = __ballot_sync(0xFFFFFFFFu, need64);
            if (ball) {
                if (need64) {
                    const int pos = rq_n + __popc(ball & ((1u << lane) - 1u));
                    rq_t[pos] = (uint32_t)t;
                    rq_kh[pos] = (uint32_t)kk | ((uint32_t)hh << 16);
                }
                rq_n += __popc(ball);
                __syncwarp();
                if (rq_n >= 32) {
                    flush_queue(A, rq_t, rq_kh, 32, &n_re);
                    const int rest = rq_n - 32;
                    uint32_t mt = 0, mkh = 0;
                    if ((int)lane < rest) { mt = rq_t[32 + lane]; mkh = rq_kh[32 + lane]; }
                    __syncwarp();
                    if ((int)lane < rest) { rq_t[lane] = mt; rq_kh[lane] = mkh; }
                    __syncwarp();
                    rq_n = rest;
                }
            }
        }
        // advance by 32 slots
        h += 32;
        while (h >= H) { h -= H; ++k; }
    }
    if (!A.list_mode) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
            rmax = fmaxf(rmax, __shfl_xor_sync(0xFFFFFFFFu, rmax, off));
            pm |= __shfl_xor_sync(0xFFFFFFFFu, pm, off);
        }
        if (lane == 0 && cnt) {
            Acc* ac = A.acc + t;
            atomicAdd(&ac->count, cnt);
            atomicMax(&ac->rmax_bits, __float_as_int(rmax));
            atomicOr(&ac->pmask, pm);
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(256) k_search(const SearchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H;
    Smem S;
    S.r = reinterpret_cast<float*>(smem);
    S.sc = reinterpret_cast<float2*>(smem + ((K * 4 + 15) & ~15));
    unsigned char* q = smem + ((K * 4 + 15) & ~15) + ((H * 8 + 15) & ~15);
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    S.rq_t = reinterpret_cast<uint32_t*>(q);
    S.rq_kh = S.rq_t + nwarps * kRqCap;
    for (int i = threadIdx.x; i < K; i += blockDim.x) S.r[i] = A.grid.r32[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) S.sc[i] = A.grid.sc32[i];
    __syncthreads();
    float Ax[3], Bz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    uint32_t* rq_t = S.rq_t + warp * kRqCap;
    uint32_t* rq_kh = S.rq_kh + warp * kRqCap;
    int rq_n = 0;
    unsigned long long n_flag = 0, n_re = 0;
    const int kchunk = A.shape.kchunk;
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
            const uint32_t fl = A.tf[t].flags;
            if (fl & 1u)
                run_item<PREC, true>(A, S, t, k0, k1, Ax, Bz, rq_t, rq_kh, rq_n, n_flag, n_re);
            else
                run_item<PREC, false>(A, S, t, k0, k1, Ax, Bz, rq_t, rq_kh, rq_n, n_flag, n_re);
        } else {
            run_item<PREC, true>(A, S, t, k0, k1, Ax, Bz, rq_t, rq_kh, rq_n, n_flag, n_re);
        }
    }
    if (PREC == CVS_PREC_FP32_RECHECK && rq_n > 0) flush_queue(A, rq_t, rq_kh, rq_n, &n_re);
    // statistics
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

// ------------------------------------------------------------ finalize
__global__ void k_finalize_colors(const Acc* __restrict__ acc, int64_t n, float* max_r,
                                  int32_t* count, uint8_t* pmask) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const Acc a = acc[t];
    max_r[t] = __int_as_float(a.rmax_bits);
    count[t] = a.count;
    pmask[t] = (uint8_t)a.pmask;
}

__global__ void k_finalize_images(const Acc* __restrict__ acc, const TargetF64* __restrict__ td,
                                  int64_t n, const ImageDesc* __restrict__ imgs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const Acc a = acc[t];
    const uint64_t slot = td[t].out_slot;
    const int i = (int)(slot >> 40);
    const int64_t local = (int64_t)(slot & ((1ull << 40) - 1));
    const ImageDesc im = imgs[i];
    im.max_r[local] = __int_as_float(a.rmax_bits);
    im.count[local] = a.count;
    im.pmask[local] = (uint8_t)a.pmask;
}

// ------------------------------------------------------------ list compaction
// One block: records with pattern != 0, in index order ((k, m) order).
__global__ void __launch_bounds__(1024) k_compact_pairs(const cvs_pair* __restrict__ dense,
                                                        int64_t n, cvs_pair* out,
                                                        unsigned long long* n_out) {
    __shared__ int warp_sums[32];
    __shared__ long long base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t start = 0; start < n; start += blockDim.x) {
        const int64_t i = start + threadIdx.x;
        const bool valid = i < n && dense[i].pattern != 0;
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, valid);
        if (lane == 0) warp_sums[warp] = __popc(ball);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) before += warp_sums[w];
            total += warp_sums[w];
        }
        if (valid) out[base + before + __popc(ball & ((1u << lane) - 1u))] = dense[i];
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = (unsigned long long)base;
}

// ------------------------------------------------------------ L*a*b* only
__global__ void k_target_lab(const uint8_t* __restrict__ rgb, int64_t n, double* lab) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double L, a, b;
    target_lab64(rgb[3 * t], rgb[3 * t + 1], rgb[3 * t + 2], L, a, b);
    lab[3 * t] = L;
    lab[3 * t + 1] = a;
    lab[3 * t + 2] = b;
}

// ------------------------------------------------------------ precision probe
// Every (target, k, m) plus-colour in FP32 and FP64: the largest |v32 - v64| of
// values within 0.05 of a rounding boundary (v in code units), the largest
// |lin32 - lin64|, and the number of FP32 codes in [-1, 256] that differ.
__global__ void k_precision_probe(const TargetF32* __restrict__ tf, const TargetF64* __restrict__ td,
                                  int64_t n, const GridDev g, const long long* __restrict__ qkey,
                                  unsigned int* max_v_err_bits, unsigned int* max_lin_err_bits,
                                  unsigned long long* n_wrong) {
    float Ax[3], Bz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    const int64_t total = n * g.K * g.N;
    float vmax = 0.0f, lmax = 0.0f;
    unsigned long long wrong = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / ((int64_t)g.K * g.N);
        const int rem = (int)(i - t * g.K * g.N);
        const int k = rem / g.N, m = rem - k * g.N;
        const TargetF32 T = tf[t];
        const TargetF64 D = td[t];
        const float r = g.r32[k];
        const float2 sc = g.sc32[m];
        int yp[3], ym[3];
        if (T.flags & 1u) codes32<true>(T, Ax, Bz, r * sc.x, r * sc.y, 0.5f, yp, ym);
        else codes32<false>(T, Ax, Bz, r * sc.x, r * sc.y, 0.5f, yp, ym);
        // FP64 reference of the plus colour
        const double da = __dmul_rn(g.r64[k], g.s64[m]), db = __dmul_rn(g.r64[k], g.c64[m]);
        double lin[3];
        color_lin64(D.L, __dadd_rn(D.a, da), __dadd_rn(D.b, db), lin);
        // FP32 plus colour, recomputed to get the unrounded values
        float dX, dZ;
        const float u = r * sc.x, w = r * sc.y;
        if (T.flags & 1u) {
            dX = u * fmaf(u, T.c1x + u, T.c2x);
            dZ = w * fmaf(w, T.c1z + w, T.c2z);
        } else {
            const float brk = (float)kFinvBreak, add = (float)kFLinAdd, mul = (float)kFinvLinMul;
            const float fx = T.fx0 + u, fz = T.fz0 + w;
            dX = (fx > brk ? fx * fx * fx : (fx - add) * mul) - T.X30;
            dZ = (fz > brk ? fz * fz * fz : (fz - add) * mul) - T.Z30;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float l32 = fmaf(Bz[c], dZ, fmaf(Ax[c], dX, T.lin0[c]));
            const float v32 = encode_v32(l32);
            const double l64 = lin[c];
            const double v64 = l64 <= 0.0031308 ? 3294.6 * l64 : 269.025 * pow(l64, 1.0 / 2.4) - 14.025;
            lmax = fmaxf(lmax, (float)fabs((double)l32 - l64));
            const double frac = v64 - floor(v64);
            if (fabs(frac - 0.5) < 0.05 && v64 > -2.0 && v64 < 258.0)
                vmax = fmaxf(vmax, (float)fabs((double)v32 - v64));
            const int q64 = quantize64(l64, qkey);
            const int q32 = (int)fminf(fmaxf(rintf(v32), -1.0f), 256.0f);
            if (q64 != q32 && q64 >= 0 && q64 <= 255) ++wrong;
        }
        (void)yp;
        (void)ym;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        vmax = fmaxf(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, off));
        lmax = fmaxf(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, off));
        wrong += __shfl_xor_sync(0xFFFFFFFFu, wrong, off);
    }
    if (lane_id() == 0) {
        atomicMax(max_v_err_bits, __float_as_uint(vmax));
        atomicMax(max_lin_err_bits, __float_as_uint(lmax));
        if (wrong) atomicAdd(n_wrong, wrong);
    }
}

__global__ void k_qkeys(long long* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 257) dst[i] = dkey(g_qthr[i]);
}

inline int blocks_for(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_trig_table(const double* angles_dev, int n, double* s64, double* c64,
                              float2* sc32, int* status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_trig_table<<<blocks_for(n, 128), 128, 0, st>>>(angles_dev, n, s64, c64, sc32, status);
    return cudaGetLastError();
}

cudaError_t launch_setup_colors(const uint8_t* rgb, int64_t n, double rmax, TargetF32* tf,
                                TargetF64* td, Acc* acc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_setup_colors<<<blocks_for(n, 128), 128, 0, st>>>(rgb, n, rmax, tf, td, acc);
    return cudaGetLastError();
}

cudaError_t launch_setup_images(const ImageDesc* imgs, int n_imgs, int64_t total, double rmax,
                                TargetF32* tf, TargetF64* td, Acc* acc, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    k_setup_images<<<blocks_for(total, 128), 128, 0, st>>>(imgs, n_imgs, total, rmax, tf, td, acc);
    return cudaGetLastError();
}

int search_smem_bytes(const GridDev& g, int block) {
    return ((g.K * 4 + 15) & ~15) + ((g.H * 8 + 15) & ~15) + (block / 32) * kRqCap * 8;
}

const void* search_kernel_ptr(int prec, int list_mode) {
    (void)list_mode;
    return prec == CVS_PREC_FP64 ? (const void*)k_search<CVS_PREC_FP64>
                                 : (const void*)k_search<CVS_PREC_FP32_RECHECK>;
}

cudaError_t launch_search(const SearchArgs& a, cudaStream_t st) {
    const int smem = search_smem_bytes(a.grid, a.shape.block);
    const void* fn = search_kernel_ptr(a.prec, a.list_mode);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = a.shape.blocks_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, a.shape.block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const int grid = a.num_sms * per_sm;
    if (a.prec == CVS_PREC_FP64)
        k_search<CVS_PREC_FP64><<<grid, a.shape.block, smem, st>>>(a);
    else
        k_search<CVS_PREC_FP32_RECHECK><<<grid, a.shape.block, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize_colors(const Acc* acc, int64_t n, float* max_r, int32_t* count,
                                   uint8_t* pmask, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_finalize_colors<<<blocks_for(n, 256), 256, 0, st>>>(acc, n, max_r, count, pmask);
    return cudaGetLastError();
}

cudaError_t launch_finalize_images(const Acc* acc, const TargetF64* td, int64_t n,
                                   const ImageDesc* imgs, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_finalize_images<<<blocks_for(n, 256), 256, 0, st>>>(acc, td, n, imgs);
    return cudaGetLastError();
}

cudaError_t launch_compact_pairs(const cvs_pair* dense, int64_t n_dense, cvs_pair* out,
                                 unsigned long long* n_out, cudaStream_t st) {
    k_compact_pairs<<<1, 1024, 0, st>>>(dense, n_dense, out, n_out);
    return cudaGetLastError();
}

cudaError_t launch_target_lab(const uint8_t* rgb, int64_t n, double* lab, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_target_lab<<<blocks_for(n, 128), 128, 0, st>>>(rgb, n, lab);
    return cudaGetLastError();
}

cudaError_t launch_precision_probe(const TargetF32* tf, const TargetF64* td, int64_t n,
                                   const GridDev& g, const long long* qkey,
                                   unsigned int* max_v_err_bits, unsigned int* max_lin_err_bits,
                                   unsigned long long* n_wrong, int num_sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_precision_probe<<<num_sms * 8, 256, 0, st>>>(tf, td, n, g, qkey, max_v_err_bits,
                                                    max_lin_err_bits, n_wrong);
    return cudaGetLastError();
}

cudaError_t copy_qkeys_to(long long* dst, cudaStream_t st) {
    k_qkeys<<<1, 288, 0, st>>>(dst);
    return cudaGetLastError();
}

size_t target_f32_size() { return sizeof(TargetF32); }
size_t target_f64_size() { return sizeof(TargetF64); }

void chain_constants(float Ax[3], float Bz[3]) {
    const double MI[9] = CVS_MI_INIT;
    const double W[3] = CVS_W_INIT;
    for (int c = 0; c < 3; ++c) {
        Ax[c] = (float)(MI[3 * c] * W[0]);
        Bz[c] = (float)(MI[3 * c + 2] * W[2]);
    }
}

}  // namespace cvs
