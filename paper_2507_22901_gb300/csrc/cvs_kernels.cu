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
// f-space, as biased integers y = kMagicBits + q.  The plus and minus colours
// run the same chain, so they travel as one float2 through the packed FP32x2
// instructions (component-wise IEEE round-to-nearest, as the scalar ops).
// Returns true if some code's unrounded value lies within W of a rounding
// boundary.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Per-target constants duplicated into (plus, minus) pairs, built once per
// work item so that the packed instructions find their operands paired.
struct PairsT {
    float2 c1x, c2x, c1z, c2z;
    float2 fx0, fz0, X30, Z30;
    float2 lin0[3];
};
struct PairsC {
    float2 Ax[3], Bz[3];
};

__device__ __forceinline__ PairsT make_pairs(const TargetF32& T) {
    PairsT P;
    P.c1x = dup(T.c1x);
    P.c2x = dup(T.c2x);
    P.c1z = dup(T.c1z);
    P.c2z = dup(T.c2z);
    P.fx0 = dup(T.fx0);
    P.fz0 = dup(T.fz0);
    P.X30 = dup(T.X30);
    P.Z30 = dup(T.Z30);
#pragma unroll
    for (int c = 0; c < 3; ++c) P.lin0[c] = dup(T.lin0[c]);
    return P;
}

__device__ __forceinline__ PairsC make_pairs(const ChainF32& C) {
    PairsC P;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        P.Ax[c] = dup(C.Ax[c]);
        P.Bz[c] = dup(C.Bz[c]);
    }
    return P;
}

// f^-1 displacement of X and Z for the pair: u2 = (u, -u), w2 = (w, -w).
template <bool FAST>
__device__ __forceinline__ void delta_xz(const PairsT& P, float2 u2, float2 w2, float2& dX,
                                         float2& dZ) {
    if (FAST) {
        // (f0 + u)^3 - f0^3 = u (3 f0^2 + u (3 f0 + u)), for +u and -u at once
        dX = __fmul2_rn(u2, __ffma2_rn(u2, __fadd2_rn(P.c1x, u2), P.c2x));
        dZ = __fmul2_rn(w2, __ffma2_rn(w2, __fadd2_rn(P.c1z, w2), P.c2z));
    } else {
        const float brk = (float)kFinvBreak, add = (float)kFLinAdd, mul = (float)kFinvLinMul;
        const float2 fx = __fadd2_rn(P.fx0, u2), fz = __fadd2_rn(P.fz0, w2);
        const float2 cx = __fmul2_rn(__fmul2_rn(fx, fx), fx), cz = __fmul2_rn(__fmul2_rn(fz, fz), fz);
        const float2 lx = __fmul2_rn(__fadd2_rn(fx, dup(-add)), dup(mul));
        const float2 lz = __fmul2_rn(__fadd2_rn(fz, dup(-add)), dup(mul));
        dX = __fadd2_rn(f2(fx.x > brk ? cx.x : lx.x, fx.y > brk ? cx.y : lx.y), neg2(P.X30));
        dZ = __fadd2_rn(f2(fz.x > brk ? cz.x : lz.x, fz.y > brk ? cz.y : lz.y), neg2(P.Z30));
    }
}

// Codes of the pair as biased integers y = kMagicBits + q.  The plus and minus
// colours run the same chain, so they travel as one float2 through the packed
// FP32x2 instructions (component-wise IEEE round-to-nearest, as the scalar
// ops).  Returns true if some code's unrounded value lies within W of a
// rounding boundary.  LINSEG = false when every linear RGB value of the call
// is known to lie above the sRGB linear segment (see pow_branch_only).
template <bool FAST, bool LINSEG = true>
__device__ __forceinline__ bool codes32(const PairsT& P, const PairsC& C, float2 u2, float2 w2,
                                        float half_w, int yp[3], int ym[3]) {
    float2 dX, dZ;
    delta_xz<FAST>(P, u2, w2, dX, dZ);
    bool flag = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 lin = __ffma2_rn(C.Bz[c], dZ, __ffma2_rn(C.Ax[c], dX, P.lin0[c]));
        float lgp, lgm, pp, pm;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lgp) : "f"(lin.x));
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lgm) : "f"(lin.y));
        const float2 e = __fmul2_rn(f2(lgp, lgm), dup(5.0f / 12.0f));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(pp) : "f"(e.x));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(pm) : "f"(e.y));
        const float2 vpow = __ffma2_rn(dup(269.025f), f2(pp, pm), dup(-14.025f));
        float2 v = vpow;
        if (LINSEG) {
            const float2 vlin = __fmul2_rn(lin, dup(3294.6f));
            v = f2(lin.x <= 0.0031308f ? vlin.x : vpow.x, lin.y <= 0.0031308f ? vlin.y : vpow.y);
        }
        const float2 y = __fadd2_rn(v, dup(kMagic));
        const float2 rr = __fadd2_rn(y, dup(-kMagic));
        const float2 d = __ffma2_rn(rr, dup(-1.0f), v);  // v - rr, exact
        flag |= fabsf(d.x) >= half_w;
        flag |= fabsf(d.y) >= half_w;
        yp[c] = __float_as_int(y.x);
        ym[c] = __float_as_int(y.y);
    }
    return flag;
}

// True when no candidate at radius r (any angle) of a fast-path target can
// reach the linear segment of the sRGB encode (lin <= 0.0031308).  The f^-1
// displacement u (c2 + u (c1 + u)) increases with u, so per channel the
// smallest linear value over |u| <= r/500, |w| <= r/200 sits at an end of
// each range.  The margin (2e-5) is far above the FP32 chain's error in
// linear RGB (below 1e-6) and the rounding of this bound.
__device__ __forceinline__ bool pow_branch_only(const TargetF32& T, const ChainF32& C, float r) {
    const float U = r * 0.002f * 1.00001f, V = r * 0.005f * 1.00001f;
    const float xlo = -U * (T.c2x - U * (T.c1x - U)), xhi = U * (T.c2x + U * (T.c1x + U));
    const float zlo = -V * (T.c2z - V * (T.c1z - V)), zhi = V * (T.c2z + V * (T.c1z + V));
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float g = T.lin0[c] + fminf(C.Ax[c] * xlo, C.Ax[c] * xhi) +
                        fminf(C.Bz[c] * zlo, C.Bz[c] * zhi);
        ok = ok && g > 0.0031308f + 2e-5f;
    }
    return ok;
}

// First radius index in [k0, k1) whose candidates may reach the sRGB linear
// segment (k1 if none); warp-uniform.
__device__ __forceinline__ int first_linseg_radius(const TargetF32& T, const ChainF32& C,
                                                   const float2* r2s, int k0, int k1) {
    const unsigned lane = threadIdx.x & 31u;
    for (int kb = k0; kb < k1; kb += 32) {
        const int kk = kb + (int)lane;
        const bool bad = kk < k1 && !pow_branch_only(T, C, r2s[kk].x);
        const unsigned b = __ballot_sync(0xFFFFFFFFu, bad);
        if (b) return kb + __ffs(b) - 1;
    }
    return k1;
}

// Embedding-signal decision on biased codes y = kMagicBits + q (exact when no
// code is flagged).  Per channel the difference d = q+ - q- indexes a 512-entry
// table in shared memory (index d & 511): bit 3 = neither high nor low, bit
// (2 - c) = high.  OR-ing the three channels gives the pattern in bits 0..2 and
// "invalid" in bit 3; okmask has bit p set for each enabled pattern p.
// Gamut (reject): all six codes lie in [0, 255] exactly when the OR of the
// six y, XOR kMagicBits, is at most 255 (every |q| here is far below 2^22).
template <bool CLIP>
__device__ __forceinline__ int decide32(const int yp_in[3], const int ym_in[3],
                                        const uint8_t* __restrict__ lut, uint32_t okmask) {
    int yp[3], ym[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        yp[c] = yp_in[c];
        ym[c] = ym_in[c];
        if (CLIP) {
            yp[c] = min(max(yp[c], kMagicBits), kMagicBits + 255);
            ym[c] = min(max(ym[c], kMagicBits), kMagicBits + 255);
        }
    }
    bool in_gamut = true;
    if (!CLIP) {
        const uint32_t o = ((uint32_t)yp[0] | (uint32_t)ym[0] | (uint32_t)yp[1]) |
                           ((uint32_t)ym[1] | (uint32_t)yp[2] | (uint32_t)ym[2]);
        in_gamut = (o ^ (uint32_t)kMagicBits) <= 255u;
    }
    uint32_t comb = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) comb |= lut[c * 512 + ((yp[c] - ym[c]) & 511)];
    const bool ok = in_gamut && ((okmask >> comb) & 1u);
    return ok ? (int)(comb & 7u) : 0;
}

// Build the three 512-entry channel tables of decide32 in shared memory.
__device__ __forceinline__ void build_decide_lut(uint8_t* lut, int32_t hi_min, int32_t lo_max) {
    for (int i = threadIdx.x; i < 3 * 512; i += blockDim.x) {
        const int c = i >> 9, idx = i & 511;
        const int d = idx < 256 ? idx : idx - 512;  // idx = d & 511 for d in [-256, 255]
        const int ad = d < 0 ? -d : d;
        uint8_t e;
        if (ad > 255) e = 8;  // cannot happen for codes in [0, 255]
        else {
            const bool hi = ad >= hi_min, lo = ad <= lo_max;
            e = (uint8_t)((hi ? (1u << (2 - c)) : 0u) | ((hi || lo) ? 0u : 8u));
        }
        lut[i] = e;
    }
}

// Exact analysis of a slot with flagged codes: each flagged code may be one
// off towards its nearby boundary.  intervals32 recomputes the slot (operation
// for operation as codes32) and bounds every code; certain_from decides a
// threshold set from the bounds: -1 = re-decide in FP64, else the exact
// pattern (0 = fail).
struct Intervals {
    int lo[6], hi[6];  // values 0..2 plus colour, 3..5 minus colour
    bool any_flag;
};

template <bool FAST>
__device__ __noinline__ Intervals intervals32(const TargetF32 T, const ChainF32 C, float u,
                                              float w, float half_w, int32_t clip) {
    const PairsT P = make_pairs(T);
    const PairsC PC = make_pairs(C);
    float2 dX2, dZ2;
    delta_xz<FAST>(P, f2(u, -u), f2(w, -w), dX2, dZ2);
    Intervals I;
    I.any_flag = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 lin2 = __ffma2_rn(PC.Bz[c], dZ2, __ffma2_rn(PC.Ax[c], dX2, P.lin0[c]));
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float lin = s ? lin2.y : lin2.x;
            const float v = encode_v32(lin);
            const float rr = __fsub_rn(__fadd_rn(v, kMagic), kMagic);
            const int q = (int)rr;
            const float d = __fsub_rn(v, rr);
            const bool f = fabsf(d) >= half_w;
            I.any_flag |= f;
            const int j = 3 * s + c;
            I.lo[j] = q - ((f && d < 0.0f) ? 1 : 0);
            I.hi[j] = q + ((f && d >= 0.0f) ? 1 : 0);
            if (clip) {
                I.lo[j] = min(max(I.lo[j], 0), 255);
                I.hi[j] = min(max(I.hi[j], 0), 255);
            }
        }
    }
    return I;
}

__device__ __forceinline__ int certain_from(const Intervals& I, int32_t hi_min, int32_t lo_max,
                                            uint32_t mask2, int32_t clip, int list_mode) {
    bool certain_out = false, maybe_out = false;
    if (!clip) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            certain_out |= I.hi[j] < 0 || I.lo[j] > 255;
            maybe_out |= I.lo[j] < 0 || I.hi[j] > 255;
        }
    }
    if (certain_out) return 0;
    bool certain_invalid = false, unstable = maybe_out;
    int pattern = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int dmax = max(I.hi[c] - I.lo[3 + c], I.hi[3 + c] - I.lo[c]);
        const int dmin = max(0, max(I.lo[c] - I.hi[3 + c], I.lo[3 + c] - I.hi[c]));
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
    if (ok && list_mode && I.any_flag) return -1;
    return ok ? pattern : 0;
}

template <bool FAST>
__device__ __noinline__ int certain32(const TargetF32 T, const ChainF32 C, float u, float w,
                                      float half_w, int32_t hi_min, int32_t lo_max,
                                      uint32_t mask2, int32_t clip, int list_mode) {
    const Intervals I = intervals32<FAST>(T, C, u, w, half_w, clip);
    return certain_from(I, hi_min, lo_max, mask2, clip, list_mode);
}

// ------------------------------------------------------------ search kernel
struct Smem {
    float2* r2;     // K: (r, r)
    float4* sc4;    // H: (sin/500, -sin/500, -cos/200, cos/200)
    uint8_t* lut;   // 3 x 512 channel-difference classes
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

// Queue up to 32 slots for FP64 re-decision; flush when 32 are waiting.
__device__ __forceinline__ void push_fp64(const SearchArgs& A, bool need64, int64_t t, int k,
                                          int h, uint32_t* rq_t, uint32_t* rq_kh, int& rq_n,
                                          unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, need64);
    if (!ball) return;
    if (need64) {
        const int pos = rq_n + __popc(ball & ((1u << lane) - 1u));
        rq_t[pos] = (uint32_t)t;
        rq_kh[pos] = (uint32_t)k | ((uint32_t)h << 16);
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

// Decide up to 32 flagged slots of target t, one per lane: exact interval
// analysis in FP32, FP64 re-decision where the analysis cannot decide.
template <bool FAST>
__device__ __forceinline__ void drain_flagged(const SearchArgs& A, const Smem& S,
                                              const TargetF32& T, const ChainF32& C, int64_t t,
                                              uint32_t* pq, int n, int& cnt, float& rmax,
                                              uint32_t& pm, uint32_t* rq_t, uint32_t* rq_kh,
                                              int& rq_n, unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int inc = A.grid.sym ? 2 : 1;
    int k = 0, h = 0, pc = 0;
    if ((int)lane < n) {
        const uint32_t kh = pq[lane];
        k = (int)(kh & 0xFFFFu);
        h = (int)(kh >> 16);
        const float r = S.r2[k].x;
        const float4 sc = S.sc4[h];
        pc = certain32<FAST>(T, C, r * sc.x, r * sc.z, A.half_w, A.hi_min, A.lo_max, A.mask2,
                             A.clip, A.list_mode);
        if (pc > 0) {
            cnt += inc;
            rmax = fmaxf(rmax, r);
            pm |= 1u << pc;
        }
    }
    __syncwarp();
    push_fp64(A, (int)lane < n && pc < 0, t, k, h, rq_t, rq_kh, rq_n, n_re);
}

// Per-lane accumulators of one work item.
struct Tally {
    int cnt;
    float rmax;
    uint32_t pm;
};

// One 32-slot step of a work item: every lane evaluates slot (k, h).  With
// CHECK, lanes past the item's last slot (active == false) contribute nothing.
// Returns true for a flagged FP32 slot (decided later by drain_flagged); the
// step itself never synchronises the warp.
template <int PREC, bool FAST, bool CHECK, bool CLIP, bool LIST, bool LINSEG>
__device__ __forceinline__ bool slot_step(const SearchArgs& A, const Smem& S, const PairsT& P,
                                          const PairsC& PC, const TargetF64& D, int k, int h,
                                          bool active, Tally& acc) {
    const int H = A.grid.H;
    const int inc = A.grid.sym ? 2 : 1;
    if (CHECK && !active) { k = 0; h = 0; }
    const float2 r2 = S.r2[k];
    const float r = r2.x;
    if (PREC == CVS_PREC_FP32_RECHECK) {
        const float4 sc = S.sc4[h];
        const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y));  // (u, -u)
        const float2 w2 = __fmul2_rn(r2, f2(sc.z, sc.w));  // (w, -w)
        int yp[3], ym[3];
        bool flag = codes32<FAST, LINSEG>(P, PC, u2, w2, A.half_w, yp, ym);
        if (CHECK) flag = flag && active;
        int pattern = decide32<CLIP>(yp, ym, S.lut, A.mask2);
        if (flag || (CHECK && !active)) pattern = 0;
        if (pattern) {
            if (!LIST) {
                acc.cnt += inc;
                acc.rmax = fmaxf(acc.rmax, r);
                acc.pm |= 1u << pattern;  // bit p for pattern p; shifted down at the end
            } else {
                int qp[3], qm[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int a = yp[c] - kMagicBits, b = ym[c] - kMagicBits;
                    if (CLIP) { a = min(max(a, 0), 255); b = min(max(b, 0), 255); }
                    qp[c] = a;
                    qm[c] = b;
                }
                write_records(A.dense, A.grid.N, H, A.grid.sym, k, h, qp, qm, pattern, 0u,
                              A.target_id);
            }
        }
        return flag;
    } else {
        int qp[3], qm[3];
        const int pattern = (!CHECK || active) ? decide64_slot(A, D, k, h, qp, qm) : 0;
        if (pattern) {
            if (LIST) {
                write_records(A.dense, A.grid.N, H, A.grid.sym, k, h, qp, qm, pattern, 0u,
                              A.target_id);
            } else {
                acc.cnt += inc;
                acc.rmax = fmaxf(acc.rmax, r);
                acc.pm |= 1u << pattern;
            }
        }
        return false;
    }
}

// Flag bitmap of the FP32 path: the main loop records which slots were
// flagged, one bit per (iteration, lane), in kFlagWords words per lane of a
// per-warp shared array (word w of lane l at [w * 32 + l]); bit j of word w is
// iteration seg0 + 32 w + j.  The loop itself thus carries no warp vote and no
// branch for flagged slots; collect_flagged compacts them after each segment.
constexpr int kFlagWords = 8;
constexpr int kSegIters = 32 * kFlagWords;

// Iterations [it, end) of an item (within one segment starting at seg0), with
// lanes at slot (k, h); flagged slots set their bits in fb.
template <int PREC, bool FAST, bool CHECK, bool CLIP, bool LIST, bool LINSEG>
__device__ __forceinline__ void run_range(const SearchArgs& A, const Smem& S, const PairsT& P,
                                          const PairsC& PC, const TargetF64& D, int& it, int end,
                                          int seg0, int nslots, int q32, int r32, int& k, int& h,
                                          Tally& acc, uint32_t* fb) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    while (it < end) {
        const int w = (it - seg0) >> 5;
        const int wend = min(end, seg0 + 32 * (w + 1));
        uint32_t bits = 0, bit = 1u << ((it - seg0) & 31);
        for (; it < wend; ++it) {
            const bool active = !CHECK || it * 32 + (int)lane < nslots;
            const bool flag = slot_step<PREC, FAST, CHECK, CLIP, LIST, LINSEG>(A, S, P, PC, D, k, h,
                                                                             active, acc);
            if (PREC == CVS_PREC_FP32_RECHECK && flag) bits |= bit;
            bit <<= 1;
            h += r32;
            k += q32;
            const bool wrap = h >= H;
            h = wrap ? h - H : h;
            k = wrap ? k + 1 : k;
        }
        if (PREC == CVS_PREC_FP32_RECHECK) fb[w * 32 + lane] |= bits;
    }
}

// Queue the flagged slots of one segment (words [0, nwords) of fb) into pq,
// 32 at a time, deciding each full batch with drain_flagged.
template <bool FAST>
__device__ __forceinline__ void collect_flagged(const SearchArgs& A, const Smem& S,
                                                const TargetF32& T, const ChainF32& C, int64_t t,
                                                int k0, int seg0, int nwords, uint32_t* fb,
                                                uint32_t* pq, int& pq_n, Tally& acc,
                                                uint32_t* rq_t, uint32_t* rq_kh, int& rq_n,
                                                unsigned long long& n_flag,
                                                unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    for (int w = 0; w < nwords; ++w) {
        uint32_t bits = fb[w * 32 + lane];
        fb[w * 32 + lane] = 0u;
        while (true) {
            const bool has = bits != 0u;
            const unsigned ball = __ballot_sync(0xFFFFFFFFu, has);
            if (!ball) break;
            if (has) {
                const int j = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int i = (seg0 + 32 * w + j) * 32 + (int)lane;  // slot index in the item
                const int dk = i / H;
                pq[pq_n + __popc(ball & ((1u << lane) - 1u))] =
                    (uint32_t)(k0 + dk) | ((uint32_t)(i - dk * H) << 16);
                ++n_flag;
            }
            pq_n += __popc(ball);
            __syncwarp();
            if (pq_n >= 32) {
                drain_flagged<FAST>(A, S, T, C, t, pq, 32, acc.cnt, acc.rmax, acc.pm, rq_t, rq_kh,
                                    rq_n, n_re);
                const int rest = pq_n - 32;
                const uint32_t mv = (int)lane < rest ? pq[32 + lane] : 0u;
                __syncwarp();
                if ((int)lane < rest) pq[lane] = mv;
                __syncwarp();
                pq_n = rest;
            }
        }
    }
}

template <int PREC, bool FAST, bool CLIP, bool LIST>
__device__ __forceinline__ void run_item(const SearchArgs& A, const Smem& S, int64_t t, int k0,
                                         int k1, const ChainF32& C, uint32_t* pq, uint32_t* fb,
                                         uint32_t* rq_t, uint32_t* rq_kh, int& rq_n,
                                         unsigned long long& n_flag, unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    const int nslots = (k1 - k0) * H;
    TargetF32 T;
    TargetF64 D;
    if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
    else D = A.td[t];
    const PairsT P = make_pairs(T);
    const PairsC PC = make_pairs(C);
    Tally acc{0, -1.0f, 0u};
    int pq_n = 0;  // flagged slots waiting for drain_flagged (warp-uniform)
    // slot i of the item is (k0 + i / H, i % H); lanes start at i = lane and
    // step by 32 = q32 H + r32, so one conditional wrap keeps h in [0, H)
    const int q32 = 32 / H, r32 = 32 - q32 * H;
    int k = k0 + (int)lane / H, h = (int)lane % H;
    const int nfull = nslots >> 5, nit = (nslots + 31) >> 5;
    // iterations below it_pow never reach the sRGB linear segment
    int it_pow = 0;
    if constexpr (PREC == CVS_PREC_FP32_RECHECK && FAST) {
        const int k_split = first_linseg_radius(T, C, S.r2, k0, k1);
        it_pow = k_split == k1 ? nit : ((k_split - k0) * H) >> 5;
    }
    int it = 0;
    for (int seg0 = 0; seg0 < nit; seg0 += kSegIters) {
        const int seg1 = min(seg0 + kSegIters, nit);
        const int full_end = min(seg1, nfull);
        if constexpr (PREC == CVS_PREC_FP32_RECHECK && FAST) {
            run_range<PREC, FAST, false, CLIP, LIST, false>(A, S, P, PC, D, it, min(full_end, it_pow),
                                                            seg0, nslots, q32, r32, k, h, acc, fb);
        }
        run_range<PREC, FAST, false, CLIP, LIST, true>(A, S, P, PC, D, it, full_end, seg0, nslots,
                                                       q32, r32, k, h, acc, fb);
        if (it < seg1) {  // the item's last, partial iteration
            if (PREC == CVS_PREC_FP32_RECHECK && FAST && it < it_pow)
                run_range<PREC, FAST, true, CLIP, LIST, false>(A, S, P, PC, D, it, seg1, seg0,
                                                               nslots, q32, r32, k, h, acc, fb);
            else
                run_range<PREC, FAST, true, CLIP, LIST, true>(A, S, P, PC, D, it, seg1, seg0,
                                                              nslots, q32, r32, k, h, acc, fb);
        }
        if (PREC == CVS_PREC_FP32_RECHECK) {
            __syncwarp();
            collect_flagged<FAST>(A, S, T, C, t, k0, seg0, (seg1 - seg0 + 31) >> 5, fb, pq, pq_n,
                                  acc, rq_t, rq_kh, rq_n, n_flag, n_re);
        }
    }
    if (PREC == CVS_PREC_FP32_RECHECK && pq_n > 0)
        drain_flagged<FAST>(A, S, T, C, t, pq, pq_n, acc.cnt, acc.rmax, acc.pm, rq_t, rq_kh, rq_n,
                            n_re);
    if (!LIST) {
        int cnt = acc.cnt;
        float rmax = acc.rmax;
        uint32_t pm = acc.pm;
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
            atomicOr(&ac->pmask, pm >> 1);  // bit p-1 for pattern p
        }
    }
}

// Launch bounds of the search kernel: blocks of up to CVS_SEARCH_MAX_THREADS
// threads, at least CVS_SEARCH_MIN_BLOCKS of them resident per SM.
#ifndef CVS_SEARCH_MAX_THREADS
#define CVS_SEARCH_MAX_THREADS kSearchBlock
#endif
#ifndef CVS_SEARCH_MIN_BLOCKS
#define CVS_SEARCH_MIN_BLOCKS 5
#endif

template <int PREC, bool CLIP, bool LIST>
__global__ void __launch_bounds__(CVS_SEARCH_MAX_THREADS, CVS_SEARCH_MIN_BLOCKS)
    k_search(const SearchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H;
    Smem S;
    S.r2 = reinterpret_cast<float2*>(smem);
    S.sc4 = reinterpret_cast<float4*>(smem + ((K * 8 + 15) & ~15));
    S.lut = smem + ((K * 8 + 15) & ~15) + H * 16;
    unsigned char* q = S.lut + 3 * 512;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    S.rq_t = reinterpret_cast<uint32_t*>(q);
    S.rq_kh = S.rq_t + nwarps * kRqCap;
    uint32_t* pq = S.rq_kh + nwarps * kRqCap + warp * kRqCap;
    uint32_t* fb = S.rq_kh + 2 * nwarps * kRqCap + warp * (kFlagWords * 32);
    for (int w = 0; w < kFlagWords; ++w) fb[w * 32 + lane_id()] = 0u;
    build_decide_lut(S.lut, A.hi_min, A.lo_max);
    for (int i = threadIdx.x; i < K; i += blockDim.x) S.r2[i] = dup(A.grid.r32[i]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        const float2 sc = A.grid.sc32[i];
        S.sc4[i] = make_float4(sc.x, -sc.x, sc.y, -sc.y);
    }
    __syncthreads();
    ChainF32 C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C.Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        C.Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
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
                run_item<PREC, true, CLIP, LIST>(A, S, t, k0, k1, C, pq, fb, rq_t, rq_kh, rq_n, n_flag,
                                                 n_re);
            else
                run_item<PREC, false, CLIP, LIST>(A, S, t, k0, k1, C, pq, fb, rq_t, rq_kh, rq_n, n_flag,
                                                  n_re);
        } else {
            run_item<PREC, true, CLIP, LIST>(A, S, t, k0, k1, C, pq, fb, rq_t, rq_kh, rq_n, n_flag,
                                             n_re);
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
            I = intervals32<FAST>(T, C, r * sc.x, r * sc.z, A.half_w, CLIP ? 1 : 0);
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
    if (PREC == CVS_PREC_FP32_RECHECK && FAST) {
        const int k_split = first_linseg_radius(T, C, r2s, k0, k1);
        it_pow = k_split == k1 ? nit : ((k_split - k0) * H) >> 5;
    }
    for (int it = 0; it < nit; ++it) {
        const bool active = it * 32 + (int)lane < nslots;
        const int kk = active ? k : k0, hh = active ? h : 0;
        const float2 r2 = r2s[kk];
        int yp[3], ym[3], qp[3], qm[3];
        bool flag = false;
        if (PREC == CVS_PREC_FP32_RECHECK) {
            const float4 sc = sc4s[hh];
            const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y)), w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
            if (it < it_pow) flag = codes32<FAST, false>(P, PC, u2, w2, A.half_w, yp, ym);
            else flag = codes32<FAST, true>(P, PC, u2, w2, A.half_w, yp, ym);
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
__global__ void __launch_bounds__(CVS_SEARCH_MAX_THREADS) k_search_multi(const MultiArgs A) {
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
                                  unsigned int* max_lab_err_bits, unsigned long long* n_wrong) {
    float Ax[3], Bz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    const int64_t total = n * g.K * g.N;
    float vmax = 0.0f, lmax = 0.0f, amax = 0.0f;
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
        const PairsT P = make_pairs(T);
        // FP64 reference of the plus colour
        const double da = __dmul_rn(g.r64[k], g.s64[m]), db = __dmul_rn(g.r64[k], g.c64[m]);
        double lin[3];
        color_lin64(D.L, __dadd_rn(D.a, da), __dadd_rn(D.b, db), lin);
        // FP32 plus colour, recomputed to get the unrounded values
        float2 dX2, dZ2;
        const float u = r * sc.x, w = r * sc.y;
        if (T.flags & 1u) delta_xz<true>(P, f2(u, -u), f2(w, -w), dX2, dZ2);
        else delta_xz<false>(P, f2(u, -u), f2(w, -w), dX2, dZ2);
        // L*a*b* the FP32 chain stands for: f-values fx0 + u and fz0 + w
        {
            const double fy = (D.L + 16.0) / 116.0;
            const double fx_exact = fy + (D.a + da) / 500.0, fz_exact = fy - (D.b + db) / 200.0;
            const double ea = 500.0 * fabs(((double)T.fx0 + (double)u) - fx_exact);
            const double eb = 200.0 * fabs(((double)T.fz0 + (double)w) - fz_exact);
            amax = fmaxf(amax, (float)fmax(ea, eb));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float l32 = __ffma2_rn(f2(Bz[c], Bz[c]), dZ2,
                                         __ffma2_rn(f2(Ax[c], Ax[c]), dX2,
                                                    f2(T.lin0[c], T.lin0[c]))).x;
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
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        vmax = fmaxf(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, off));
        lmax = fmaxf(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, off));
        amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, off));
        wrong += __shfl_xor_sync(0xFFFFFFFFu, wrong, off);
    }
    if (lane_id() == 0) {
        atomicMax(max_v_err_bits, __float_as_uint(vmax));
        atomicMax(max_lin_err_bits, __float_as_uint(lmax));
        atomicMax(max_lab_err_bits, __float_as_uint(amax));
        if (wrong) atomicAdd(n_wrong, wrong);
    }
}

// ------------------------------------------------------------ capacity table
// Colours first .. first+n-1 of the 2^24-colour space as (R, G, B) bytes,
// colour index = (R << 16) | (G << 8) | B.
__global__ void k_rgb_iota(uint8_t* __restrict__ rgb, int64_t first, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = (uint32_t)(first + i);
    rgb[3 * i] = (uint8_t)(v >> 16);
    rgb[3 * i + 1] = (uint8_t)(v >> 8);
    rgb[3 * i + 2] = (uint8_t)v;
}

// Pack per-colour results into the table: entry = (count << 32) | max_r bits.
__global__ void k_lut_pack(const Acc* __restrict__ acc, int64_t n, uint64_t* __restrict__ entry,
                           uint8_t* __restrict__ pmask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Acc a = acc[i];
    entry[i] = ((uint64_t)(uint32_t)a.count << 32) | (uint32_t)a.rmax_bits;
    pmask[i] = (uint8_t)a.pmask;
}

// Per-pixel maps of up to kGatherMaxImages images from the table, descriptors
// passed by value (no device-side table, so concurrent lookups share nothing).
// Blocks never straddle images: block b belongs to the image whose block range
// holds b.
__global__ void __launch_bounds__(kGatherBlock) k_lut_gather_images(const GatherBatch B,
                                                                    const uint64_t* __restrict__ entry,
                                                                    const uint8_t* __restrict__ pmask) {
    int i = 0;  // largest i with block_first[i] <= blockIdx.x
#pragma unroll 1
    for (int j = 1; j < B.n; ++j)
        if (B.block_first[j] <= (int64_t)blockIdx.x) i = j;
    const ImageDesc& im = B.img[i];
    const int64_t p = ((int64_t)blockIdx.x - B.block_first[i]) * blockDim.x + threadIdx.x;
    const int64_t npx = (int64_t)im.width * im.height;
    if (p >= npx) return;
    const int64_t y = p / im.width, x = p - y * im.width;
    const uint8_t* px = im.rgb + y * im.pitch + 3 * x;
    const uint32_t key = ((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | px[2];
    const uint64_t e = __ldg(entry + key);
    im.max_r[p] = __uint_as_float((uint32_t)e);
    im.count[p] = (int32_t)(e >> 32);
    im.pmask[p] = __ldg(pmask + key);
}

// Per-colour results of a colour list from the table.
__global__ void k_lut_gather_colors(const uint8_t* __restrict__ rgb, int64_t n,
                                    const uint64_t* __restrict__ entry,
                                    const uint8_t* __restrict__ pmask, float* max_r,
                                    int32_t* count, uint8_t* pm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = ((uint32_t)rgb[3 * i] << 16) | ((uint32_t)rgb[3 * i + 1] << 8) | rgb[3 * i + 2];
    const uint64_t e = __ldg(entry + key);
    max_r[i] = __uint_as_float((uint32_t)e);
    count[i] = (int32_t)(e >> 32);
    pm[i] = __ldg(pmask + key);
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
    // (r, r) pairs, angle quadruples, then per warp: FP64 queue (targets, slots)
    // and flagged queue
    return ((g.K * 8 + 15) & ~15) + g.H * 16 + 3 * 512 +
           (block / 32) * (kRqCap * 12 + kFlagWords * 32 * 4);
}

template <int PREC, bool CLIP, bool LIST>
cudaError_t launch_search_t(const SearchArgs& a, cudaStream_t st) {
    const int smem = search_smem_bytes(a.grid, a.shape.block);
    const void* fn = (const void*)k_search<PREC, CLIP, LIST>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = a.shape.blocks_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, a.shape.block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    k_search<PREC, CLIP, LIST><<<a.num_sms * per_sm, a.shape.block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_search_p(const SearchArgs& a, cudaStream_t st) {
    if (a.clip) return a.list_mode ? launch_search_t<PREC, true, true>(a, st)
                                   : launch_search_t<PREC, true, false>(a, st);
    return a.list_mode ? launch_search_t<PREC, false, true>(a, st)
                       : launch_search_t<PREC, false, false>(a, st);
}

cudaError_t launch_search(const SearchArgs& a, cudaStream_t st) {
    return a.prec == CVS_PREC_FP64 ? launch_search_p<CVS_PREC_FP64>(a, st)
                                   : launch_search_p<CVS_PREC_FP32_RECHECK>(a, st);
}

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
    k_init_acc<<<blocks_for(n, 256), 256, 0, st>>>(acc, n);
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
                                   unsigned int* max_lab_err_bits, unsigned long long* n_wrong,
                                   int num_sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_precision_probe<<<num_sms * 8, 256, 0, st>>>(tf, td, n, g, qkey, max_v_err_bits,
                                                    max_lin_err_bits, max_lab_err_bits, n_wrong);
    return cudaGetLastError();
}

cudaError_t launch_rgb_iota(uint8_t* rgb, int64_t first, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_rgb_iota<<<blocks_for(n, 256), 256, 0, st>>>(rgb, first, n);
    return cudaGetLastError();
}

cudaError_t launch_lut_pack(const Acc* acc, int64_t n, uint64_t* entry, uint8_t* pmask,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_lut_pack<<<blocks_for(n, 256), 256, 0, st>>>(acc, n, entry, pmask);
    return cudaGetLastError();
}

cudaError_t launch_lut_gather_images(const GatherBatch& b, int64_t total_blocks,
                                     const uint64_t* entry, const uint8_t* pmask, cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    k_lut_gather_images<<<(unsigned)total_blocks, kGatherBlock, 0, st>>>(b, entry, pmask);
    return cudaGetLastError();
}

cudaError_t launch_lut_gather_colors(const uint8_t* rgb, int64_t n, const uint64_t* entry,
                                     const uint8_t* pmask, float* max_r, int32_t* count,
                                     uint8_t* pm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_lut_gather_colors<<<blocks_for(n, 256), 256, 0, st>>>(rgb, n, entry, pmask, max_r, count, pm);
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
