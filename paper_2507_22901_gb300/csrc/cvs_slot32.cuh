// cvs_slot32.cuh - the FP32 slot of the colour-pair search (sm_103a), shared
// by the single-threshold and the multi-threshold search kernels.
//
// A slot is one (radius k, angle h) of a target: the point-symmetric pair
// (L*, a* +- r sin j, b* +- r cos j) of §2 Methods, converted back to 8-bit
// sRGB.  This header holds the packed FP32x2 chain (codes32), the
// table-driven embedding-signal decision (decide32), and the exact interval
// analysis of slots whose codes sit near a rounding boundary (intervals32,
// certain_from).
#pragma once

#include <cuda_runtime.h>

#include "cvs_device.cuh"
#include "cvs_internal.h"

namespace cvs {
namespace {

constexpr int kRqCap = 64;  // re-decision queue entries per warp

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

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
// Linear RGB of the pair (plus in .x, minus in .y), per channel.
template <bool FAST>
__device__ __forceinline__ void lin32(const PairsT& P, const PairsC& C, float2 u2, float2 w2,
                                      float2 lin[3]) {
    float2 dX, dZ;
    delta_xz<FAST>(P, u2, w2, dX, dZ);
#pragma unroll
    for (int c = 0; c < 3; ++c) lin[c] = __ffma2_rn(C.Bz[c], dZ, __ffma2_rn(C.Ax[c], dX, P.lin0[c]));
}

// Encode and round the pair's linear values (see codes32).
template <bool LINSEG>
__device__ __forceinline__ bool encode32(const float2 lin_in[3], float half_w, int yp[3],
                                         int ym[3], float2* resid) {
    bool flag = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 lin = lin_in[c];
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
        if (resid) resid[c] = d;  // v - round(v) of (plus, minus)
        yp[c] = __float_as_int(y.x);
        ym[c] = __float_as_int(y.y);
    }
    return flag;
}

template <bool FAST, bool LINSEG = true>
__device__ __forceinline__ bool codes32(const PairsT& P, const PairsC& C, float2 u2, float2 w2,
                                        float half_w, int yp[3], int ym[3],
                                        float2* resid = nullptr) {
    float2 lin[3];
    lin32<FAST>(P, C, u2, w2, lin);
    return encode32<LINSEG>(lin, half_w, yp, ym, resid);
}

// True when some linear value of the pair lies certainly outside the range of
// codes 0..255 (below the threshold of code 0 or at or above that of code 256,
// by a margin of 1e-5, far above the FP32 chain's error in linear RGB of about
// 1e-6): in gamut-reject mode such a pair fails whatever its codes.
constexpr double kQthrHost[257] = CVS_QTHR_INIT;
constexpr float kLinOutLo = (float)kQthrHost[0] - 1e-5f;
constexpr float kLinOutHi = (float)kQthrHost[256] + 1e-5f;
__device__ __forceinline__ bool surely_out32(const float2 lin[3]) {
    constexpr float mid = 0.5f * (kLinOutLo + kLinOutHi), half = 0.5f * (kLinOutHi - kLinOutLo);
    bool out = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 dv = __fadd2_rn(lin[c], dup(-mid));
        out |= fabsf(dv.x) > half;
        out |= fabsf(dv.y) > half;
    }
    return out;
}

// Lower bound of channel c's linear value over the pair's two colours at any
// angle, for displacements up to U = r/500 and V = r/200 (with margins), of a
// fast-path target: the larger of two bounds.  The f^-1 displacement
// u (c2 + u (c1 + u)) increases with u, so the X and Z terms are each smallest
// at an end of their range; and since u = U sin j and w = -V cos j move
// together, their linear parts form a sinusoid of amplitude
// sqrt((Ax c2x U)^2 + (Bz c2z V)^2), the quadratic parts are at least
// min(0, Ax c1x) U^2 and min(0, Bz c1z) V^2 and the cubic parts at least
// -|Ax| U^3 and -|Bz| V^3.
__device__ __forceinline__ float lin_lower_bound(const TargetF32& T, const ChainF32& C, float U,
                                                 float V, float xlo, float xhi, float zlo,
                                                 float zhi, int c) {
    const float ends = T.lin0[c] + fminf(C.Ax[c] * xlo, C.Ax[c] * xhi) +
                       fminf(C.Bz[c] * zlo, C.Bz[c] * zhi);
    const float p = C.Ax[c] * T.c2x * U, q = C.Bz[c] * T.c2z * V;
    const float coupled = T.lin0[c] - sqrtf(p * p + q * q) +
                          fminf(0.0f, C.Ax[c] * T.c1x) * U * U +
                          fminf(0.0f, C.Bz[c] * T.c1z) * V * V -
                          (fabsf(C.Ax[c]) * U * U * U + fabsf(C.Bz[c]) * V * V * V);
    return fmaxf(ends, coupled);
}

// True when no candidate at radius r (any angle) of a fast-path target can
// reach the linear segment of the sRGB encode (lin <= 0.0031308): every
// channel's lower bound stays above it by a margin (2e-5) far above the FP32
// chain's error in linear RGB (below 1e-6) and the rounding of the bound.
__device__ __forceinline__ bool pow_branch_only(const TargetF32& T, const ChainF32& C, float r) {
    const float U = r * 0.002f * 1.00001f, V = r * 0.005f * 1.00001f;
    const float xlo = -U * (T.c2x - U * (T.c1x - U)), xhi = U * (T.c2x + U * (T.c1x + U));
    const float zlo = -V * (T.c2z - V * (T.c1z - V)), zhi = V * (T.c2z + V * (T.c1z + V));
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        ok = ok && lin_lower_bound(T, C, U, V, xlo, xhi, zlo, zhi, c) > 0.0031308f + 2e-5f;
    return ok;
}

// Radius bound.  At radius r (any angle) no pair of a fast-path target can
// have a high channel c when its codes cannot differ by hi_min:
//   the pair's difference in linear RGB is, with u = r sin j / 500 and
//   w = -r cos j / 200,  Ax (2 c2x u + 2 u^3) + Bz (2 c2z w + 2 w^3),  whose
//   size over all angles is at most D = 2 sqrt((Ax c2x U)^2 + (Bz c2z V)^2)
//   + 2 |Ax| U^3 + 2 |Bz| V^3 (U = r/500, V = r/200);
//   both linear values are at least lo (lin_lower_bound);
//   the encode in code units, v(x) = 3294.6 x up to x = 0.0031308 and
//   269.025 x^(5/12) - 14.025 above, is increasing and concave (its slope only
//   falls), so two values no lower than lo and at most D apart encode to
//   values at most v(lo + D) - v(lo) apart, and their codes at most that plus
//   one.
// The bound is evaluated in FP32 with lo lowered by 1e-5, D raised by a
// relative 1e-4, and 0.01 code units added, far above its rounding errors.
__device__ __forceinline__ float v_enc_bound(float x) {
    return x <= 0.0031308f ? 3294.6f * x : 269.025f * exp2f(5.0f / 12.0f * log2f(x)) - 14.025f;
}

// The channels (bit 2 - c, as in a pattern) that could be high at radius r;
// the bound grows with r.
__device__ __forceinline__ uint32_t high_possible(const TargetF32& T, const ChainF32& C, float r,
                                                  int32_t hi_min) {
    const float U = r * 0.002f * 1.00001f, V = r * 0.005f * 1.00001f;
    const float xlo = -U * (T.c2x - U * (T.c1x - U)), xhi = U * (T.c2x + U * (T.c1x + U));
    const float zlo = -V * (T.c2z - V * (T.c1z - V)), zhi = V * (T.c2z + V * (T.c1z + V));
    uint32_t mask = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float ax = fabsf(C.Ax[c]), bz = fabsf(C.Bz[c]);
        const float p = ax * T.c2x * U, q = bz * T.c2z * V;
        const float dlin = (2.0f * sqrtf(p * p + q * q) + 2.0f * (ax * U * U * U + bz * V * V * V)) *
                           1.0001f;
        const float lo = lin_lower_bound(T, C, U, V, xlo, xhi, zlo, zhi, c) - 1e-5f;
        const float dv = v_enc_bound(lo + dlin) - v_enc_bound(lo) + 0.01f;
        if (!(dv + 1.001f < (float)hi_min)) mask |= 1u << (2 - c);
    }
    return mask;
}

__device__ __forceinline__ bool certain_fail_radius(const TargetF32& T, const ChainF32& C,
                                                    float r, int32_t hi_min) {
    return high_possible(T, C, r, hi_min) == 0u;
}

// First radius index in [k0, k1) whose candidates may pass (k1 if none);
// warp-uniform.
__device__ __forceinline__ int first_possible_radius(const TargetF32& T, const ChainF32& C,
                                                     const float2* r2s, int k0, int k1,
                                                     int32_t hi_min) {
    const unsigned lane = threadIdx.x & 31u;
    for (int kb = k0; kb < k1; kb += 32) {
        const int kk = kb + (int)lane;
        const bool maybe = kk < k1 && !certain_fail_radius(T, C, r2s[kk].x, hi_min);
        const unsigned b = __ballot_sync(0xFFFFFFFFu, maybe);
        if (b) return kb + __ffs(b) - 1;
    }
    return k1;
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

// ------------------------------------------------------------ angle ranges
// At radius r the pair's linear RGB, channel c, is lin0 + E(j) +- O(j) with
// u = U sin j, w = -V cos j (U = r/500, V = r/200) and, from the cubic
// expansion of f^-1 about the target,
//   O(j) = Ax (c2x u + u^3) + Bz (c2z w + w^3)       (odd part)
//   E(j) = Ax c1x u^2 + Bz c1z w^2                   (even part).
// Since sin^3 = (3 sin - sin 3j)/4 and cos^3 = (3 cos + cos 3j)/4,
//   O(j) = alpha sin j + beta cos j + rho(j),
//   alpha = Ax U (c2x + 3U^2/4), beta = -Bz V (c2z + 3V^2/4),
//   |rho| <= eps = sqrt((Ax U^3)^2 + (Bz V^3)^2) / 4,
// and E(j) = P sin^2 j + Q cos^2 j lies between P = Ax c1x U^2 and
// Q = Bz c1z V^2.  With R = |(alpha, beta)| and j0 the zero of the sinusoid,
// |O(j)| is within eps of R |sin(j - j0)|, a function of period pi.  So:
// - gamut (reject): both colours in range need |O| <= G = min(lin0 + max(P,Q)
//   - lo_out, hi_out - lin0 - min(P,Q)), i.e. |sin(j - j0)| <= (G + eps)/R:
//   an arc about j0;
// - a high channel needs codes hi_min apart, which by the concavity bound of
//   high_possible needs 2|O| >= tau = v^-1(v(lo) + hi_min - 1) - lo: outside
//   the arc |sin(j - j0)| < (tau/2 - eps)/R about j0.
// A slot can pass only inside every gamut arc and outside the "low" arc of at
// least one channel that an enabled pattern needs high.
// On a slow-path radius some f-values fall below delta = 6/29, where f^-1 is
// not the cube but its tangent line at delta: f^-1(f) = f^3 + e(f) with
// e(f) = -(delta - f)^2 (f + 2 delta) below delta and 0 above.  So each colour
// adds Ax (e(fx0 +- u) - e(fx0)) + Bz (e(fz0 +- w) - e(fz0)) to the cubic
// form, a departure D within [Dlo, Dhi] (finv_departure: e is non-positive
// and its size only grows as f falls, over the f-values of real colours at
// radii up to 32).  The bounds then widen by it: G by Dhi - lo_out and hi_out
// - Dlo on its two sides, lo by Dlo, and tau by Dhi - Dlo, since
// lin+ - lin- = 2 O + D+ - D-.  On a fast-path radius D is exactly 0 and the
// bounds are those above.  radius_ranges_body turns
// these arcs into slot-index ranges of a folded, evenly spaced grid (slot h
// at th0 + h pi/H) and intersects them by a sweep over their end points.
// Every bound carries margins far above its FP32 rounding: arguments of asin
// by a relative 1e-4, angles by 2e-4 rad, linear values by 1e-5.
constexpr int kMaxArcRanges = 4;  // more ranges fall back to the whole radius
constexpr float kArcAngleMargin = 2e-4f;

// Arc tangent of y/x in [-pi, pi] for the angle ranges, branch-free: octant
// reduction to t = min/max in [0, 1] and an odd polynomial of degree 11 in t
// (coefficients fitted here by weighted least squares on [0, 1]; largest
// error 1.8e-6 rad in FP32, two orders below kArcAngleMargin).
__device__ __forceinline__ float atan2_arc(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(fmaxf(ax, ay), 1e-30f), mn = fminf(ax, ay);
    const float t = __fdividef(mn, mx), s = t * t;
    float p = -0.01171913929283619f;
    p = fmaf(p, s, 0.052647363394498825f);
    p = fmaf(p, s, -0.1164264902472496f);
    p = fmaf(p, s, 0.19354037940502167f);
    p = fmaf(p, s, -0.33262282609939575f);
    p = fmaf(p, s, 0.9999772310256958f);
    float a = p * t;
    a = ay > ax ? 1.5707963267948966f - a : a;
    a = x < 0.0f ? 3.141592653589793f - a : a;
    return copysignf(a, y);
}

// Arc sine of x in [0, 0.9999] (callers treat larger arguments separately).
__device__ __forceinline__ float asin_arc(float x) {
    const float c2 = fmaxf(1.0f - x * x, 1e-30f);
    return atan2_arc(x, c2 * rsqrtf(c2));
}

// The encode bound v(x) of high_possible and a lower bound of its inverse
// (the x with v(x) >= y), on the approximate MUFU log and exp; callers keep
// margins far above their errors (relative 2^-21).  v steps down by about
// 0.007 code units at the segment boundary, so near it both inverse
// branches are taken.
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float v_enc_fast(float x) {
    const float pw = fmaf(269.025f, ex2_approx((5.0f / 12.0f) * lg2_approx(fmaxf(x, 1e-30f))), -14.025f);
    return x <= 0.0031308f ? 3294.6f * x : pw;
}
__device__ __forceinline__ float v_inv_fast(float y) {
    const float pw = ex2_approx(2.4f * lg2_approx(fmaxf((y + 14.025f) * (1.0f / 269.025f), 1e-30f)));
    return y <= 10.32f ? fminf(y * (1.0f / 3294.6f), pw) : pw;
}

// True when every candidate at radius r of target T stays on the cubic branch
// of f^-1 (f-values above 6/29 by a margin far above their FP32 rounding).
__device__ __forceinline__ bool fast_radius(const TargetF32& T, float r) {
    const float lim = (float)kFinvBreak * 1.00001f + 1e-6f;
    return T.fx0 - r * 0.002f * 1.00001f > lim && T.fz0 - r * 0.005f * 1.00001f > lim;
}

// Slots within circular distance `half` (index units) of centre c in
// (-H, 2H), as a circular range (start, len) over H slots; len 0 = none,
// len H = all.  Branch-free.
__device__ __forceinline__ void arc_range(float c, float half, int H, int& start, int& len) {
    const float hh = fminf(half, 0.5f * (float)H);
    const int a = (int)ceilf(c - hh), b = (int)floorf(c + hh);
    int l = b - a + 1;
    int s0 = a < 0 ? a + H : a;
    s0 = s0 >= H ? s0 - H : s0;
    const bool none = !(half >= 0.0f) || l <= 0;
    const bool all = !none && (half >= 0.5f * (float)H || l >= H);
    len = none ? 0 : (all ? H : l);
    start = (none || all) ? 0 : s0;
}

// The bounds of channel c at radius r without the arc trigonometry: the
// sinusoid (alpha, beta), the gamut ratio xg (|sin(j - j0)| <= xg inside the
// gamut arc; >= 0.9999: every angle; < 0: no pair of the radius is in gamut)
// and the low ratio xl (|sin(j - j0)| < xl: certainly not high; <= 0: no such
// angle; >= 1: every angle, also when no enabled pattern needs the channel),
// and the lower bound lo of lin_lower_bound.
struct ArcChannel {
    float alpha, beta, xg, xl, lo;
    float invR, eps, emid, ehalf, l0;  // E(j) = emid + ehalf cos 2j; the target's linear value
    float dlo, dhi;                    // the departure from the cubic, [Dlo, Dhi]
};

// Range [lo, hi] of e(f0 + d) - e(f0) over |d| <= Di (Di with its margin,
// as fast_radius takes it): exactly 0 where f0 - Di stays above delta.
struct FinvDeparture {
    float xlo, xhi, zlo, zhi;
};

__device__ __forceinline__ void finv_departure(float f0, float Di, float& lo, float& hi) {
    const float dl = (float)kFinvBreak;
    const float fmin = f0 - Di;
    if (fmin > dl * 1.00001f + 1e-6f) {
        lo = 0.0f;
        hi = 0.0f;
        return;
    }
    const float tm = fmaxf(dl - fmin, 0.0f), t0 = fmaxf(dl - f0, 0.0f);
    const float emax = tm * tm * (fmin + 2.0f * dl) * 1.0001f + 1e-7f;  // |e| at the lowest f
    const float e0 = t0 * t0 * (f0 + 2.0f * dl);                        // |e(f0)|
    lo = -emax + e0 * 0.9999f - 1e-7f;
    hi = e0 * 1.0001f + 1e-7f;
}

__device__ __forceinline__ ArcChannel channel_bounds(const TargetF32& T, const ChainF32& C, float r,
                                                     int c, int32_t hi_min, bool need_high,
                                                     bool clip, const FinvDeparture& dep) {
    const float U = r * 0.002f, V = r * 0.005f;
    const float Ui = U * 1.00001f, Vi = V * 1.00001f;
    const float ax = c == 0 ? C.Ax[0] : (c == 1 ? C.Ax[1] : C.Ax[2]);
    const float bz = c == 0 ? C.Bz[0] : (c == 1 ? C.Bz[1] : C.Bz[2]);
    const float l0 = c == 0 ? T.lin0[0] : (c == 1 ? T.lin0[1] : T.lin0[2]);
    ArcChannel o;
    o.alpha = ax * U * (T.c2x + 0.75f * U * U);
    o.beta = -bz * V * (T.c2z + 0.75f * V * V);
    const float R2 = fmaxf(o.alpha * o.alpha + o.beta * o.beta, 1e-30f);
    const float invR = rsqrtf(R2) * 1.00001f;  // 1/R, rounded up
    const float au = ax * Ui * Ui * Ui, bv = bz * Vi * Vi * Vi;
    const float e2 = fmaxf(au * au + bv * bv, 1e-36f);
    const float eps = 0.25f * e2 * rsqrtf(e2) * 1.0001f + 1e-7f;
    o.xg = 2.0f;
    o.invR = invR;
    o.eps = eps;
    o.l0 = l0;
    o.dlo = fminf(ax * dep.xlo, ax * dep.xhi) + fminf(bz * dep.zlo, bz * dep.zhi);
    o.dhi = fmaxf(ax * dep.xlo, ax * dep.xhi) + fmaxf(bz * dep.zlo, bz * dep.zhi);
    if (!clip) {
        const float P = ax * T.c1x * U * U, Q = bz * T.c1z * V * V;
        o.emid = 0.5f * (P + Q);
        o.ehalf = 0.5f * (Q - P);
        const float G = fminf(l0 + fmaxf(P, Q) + o.dhi - kLinOutLo,
                              kLinOutHi - l0 - fminf(P, Q) - o.dlo) + eps + 1e-5f;
        o.xg = G < 0.0f ? -1.0f : G * invR * 1.0001f + 1e-6f;
    }
    // the lower bound of lin_lower_bound, per channel
    const float xlo = -Ui * (T.c2x - Ui * (T.c1x - Ui)), xhi = Ui * (T.c2x + Ui * (T.c1x + Ui));
    const float zlo = -Vi * (T.c2z - Vi * (T.c1z - Vi)), zhi = Vi * (T.c2z + Vi * (T.c1z + Vi));
    const float ends = l0 + fminf(ax * xlo, ax * xhi) + fminf(bz * zlo, bz * zhi);
    const float p = ax * T.c2x * Ui, q = bz * T.c2z * Vi;
    const float pq2 = fmaxf(p * p + q * q, 1e-36f);
    const float coupled = l0 - pq2 * rsqrtf(pq2) * 1.00001f + fminf(0.0f, ax * T.c1x) * Ui * Ui +
                          fminf(0.0f, bz * T.c1z) * Vi * Vi -
                          (fabsf(ax) * Ui * Ui * Ui + fabsf(bz) * Vi * Vi * Vi);
    o.lo = fmaxf(ends, coupled) - 1e-5f + o.dlo;
    const float lo = clip ? o.lo : fmaxf(o.lo, kLinOutLo);
    const float y = v_enc_fast(lo) + (float)hi_min - 1.02f;
    const float tau = (v_inv_fast(y) - lo) * 0.9999f - 3e-6f;
    const float ostar = 0.5f * (tau - (o.dhi - o.dlo));
    o.xl = need_high ? (ostar - eps) * invR * 0.9999f - 1e-6f : 2.0f;
    return o;
}

// The gamut and low arcs of one channel as circular slot ranges (gamut start,
// len, low start, len).
__device__ __forceinline__ int4 channel_arcs(const ArcChannel& a, float th0, float inv_step, int H) {
    float cidx = (atan2_arc(-a.beta, a.alpha) - th0) * inv_step;
    cidx -= (float)H * floorf(cidx * (1.0f / (float)H));
    int4 o;
    float xg = a.xg;
    if (xg < 0.9999f) {
        // E over the gamut arc only: the arc is j0 +- w with sin w = xg, and
        // E = emid + ehalf cos 2j, cos 2j = 1 - 2 sin^2 j; cos 2j reaches 1
        // inside it where |sin j0| <= sin w, -1 where |cos j0| <= sin w.  The
        // arc from the narrower E lies inside this one, so the bound holds.
        const float invr = rsqrtf(fmaxf(a.alpha * a.alpha + a.beta * a.beta, 1e-30f));
        const float sj = -a.beta * invr, cj = a.alpha * invr;  // sin j0, cos j0
        const float sw = xg, cw = sqrtf(fmaxf(1.0f - xg * xg, 0.0f));
        const float s1 = sj * cw - cj * sw, s2 = sj * cw + cj * sw;
        const float c1 = 1.0f - 2.0f * s1 * s1, c2 = 1.0f - 2.0f * s2 * s2;
        const float cmax = fabsf(sj) <= sw + 1e-5f ? 1.0f : fminf(fmaxf(c1, c2) + 1e-5f, 1.0f);
        const float cmin = fabsf(cj) <= sw + 1e-5f ? -1.0f : fmaxf(fminf(c1, c2) - 1e-5f, -1.0f);
        const float e_a = a.ehalf * cmin, e_b = a.ehalf * cmax;
        const float emin = a.emid + fminf(e_a, e_b) - 1e-7f, emax = a.emid + fmaxf(e_a, e_b) + 1e-7f;
        const float G = fminf(a.l0 + emax + a.dhi - kLinOutLo, kLinOutHi - a.l0 - emin - a.dlo) +
                        a.eps + 1e-5f;
        xg = fminf(xg, G < 0.0f ? -1.0f : G * a.invR * 1.0001f + 1e-6f);
    }
    if (xg < 0.0f) {  // no angle of the radius keeps this channel in gamut
        o.x = 0;
        o.y = 0;
        o.z = 0;
        o.w = 0;
        return o;
    }
    const float hg = (asin_arc(fminf(xg, 0.9999f)) + kArcAngleMargin) * inv_step;
    arc_range(cidx, xg >= 0.9999f ? (float)H : hg, H, o.x, o.y);
    const float hl = (asin_arc(fminf(a.xl, 0.9999f)) - kArcAngleMargin) * inv_step;
    arc_range(cidx, a.xl >= 1.0f ? (float)H : (a.xl > 0.0f ? hl : -1.0f), H, o.z, o.w);
    return o;
}

// Feasible slot ranges of radius r for any target (on a slow-path radius
// with the bounds widened by the departure of f^-1 from its cubic): writes up to
// kMaxArcRanges entries (start | len << 16), disjoint and ascending, to out
// and returns their number; total = slots covered.  chm: channels an enabled
// pattern needs high (bit 2 - c for channel c).
template <bool CLIP>
__device__ __forceinline__ int radius_ranges_body(const TargetF32& T, const ChainF32& C, float r,
                                                  int32_t hi_min, uint32_t chm, float th0,
                                                  float inv_step, int H, uint32_t* out,
                                                  int& total) {
    FinvDeparture dep;
    finv_departure(T.fx0, r * 0.002f * 1.00001f, dep.xlo, dep.xhi);
    finv_departure(T.fz0, r * 0.005f * 1.00001f, dep.zlo, dep.zhi);
    ArcChannel ch[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        ch[c] = channel_bounds(T, C, r, c, hi_min, (chm >> (2 - c)) & 1u, CLIP, dep);
    total = 0;
    // no slot: a channel leaves the gamut at every angle, or no channel can be high
    if (ch[0].xg < 0.0f || ch[1].xg < 0.0f || ch[2].xg < 0.0f ||
        (ch[0].xl >= 1.0f && ch[1].xl >= 1.0f && ch[2].xl >= 1.0f))
        return 0;
    // every slot: in gamut at every angle and some channel free of a low arc
    if (ch[0].xg >= 0.9999f && ch[1].xg >= 0.9999f && ch[2].xg >= 0.9999f &&
        (ch[0].xl <= 0.0f || ch[1].xl <= 0.0f || ch[2].xl <= 0.0f)) {
        out[0] = (uint32_t)H << 16;
        total = H;
        return 1;
    }
    int rs[6], rl[6];  // ranges 0..2: gamut arcs, 3..5: low arcs
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int4 o = channel_arcs(ch[c], th0, inv_step, H);
        rs[c] = o.x;
        rl[c] = o.y;
        rs[3 + c] = o.z;
        rl[3 + c] = o.w;
    }
    if (rl[0] == 0 || rl[1] == 0 || rl[2] == 0) return 0;
    // membership of slot 0, and the positions (> 0) where a range is entered or left
    constexpr int kSentinel = 0x7FFFFFFF;
    uint32_t state = 0;
    int ev[12];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int s0 = rs[i], l = rl[i];
        const bool partial = l > 0 && l < H;
        if (l >= H || (partial && (s0 == 0 || s0 + l > H))) state |= 1u << i;
        const int e1 = s0 + l >= H ? s0 + l - H : s0 + l;
        ev[2 * i] = (partial && s0 > 0) ? (s0 << 3) | i : kSentinel;
        ev[2 * i + 1] = (partial && e1 > 0) ? (e1 << 3) | i : kSentinel;
    }
    // sort the 12 keys (position, range): Batcher's odd-even merge network for
    // 16 keys restricted to 12 (41 comparators; checked on all 0/1 inputs)
    constexpr int kNet[41][2] = {
        {0, 1}, {2, 3}, {0, 2}, {1, 3}, {1, 2}, {4, 5}, {6, 7}, {4, 6}, {5, 7}, {5, 6}, {0, 4},
        {2, 6}, {2, 4}, {1, 5}, {3, 7}, {3, 5}, {1, 2}, {3, 4}, {5, 6}, {8, 9}, {10, 11}, {8, 10},
        {9, 11}, {9, 10}, {0, 8}, {4, 8}, {2, 10}, {6, 10}, {2, 4}, {6, 8}, {1, 9}, {5, 9}, {3, 11},
        {7, 11}, {3, 5}, {7, 9}, {1, 2}, {3, 4}, {5, 6}, {7, 8}, {9, 10}};
#pragma unroll
    for (int q = 0; q < 41; ++q) {
        const int a = kNet[q][0], b = kNet[q][1];
        const int lo2 = min(ev[a], ev[b]), hi2 = max(ev[a], ev[b]);
        ev[a] = lo2;
        ev[b] = hi2;
    }
    // F = inside all gamut arcs and outside the low arc of some channel
    auto feasible = [](uint32_t st) { return (st & 7u) == 7u && ((~st >> 3) & 7u) != 0u; };
    bool cur = feasible(state);
    int start = 0, n = 0;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        const int key = ev[i];
        const bool valid = key != kSentinel;
        state ^= valid ? 1u << (key & 7) : 0u;
        const int pos = key >> 3;
        const bool last = i == 11 || (ev[i + 1 < 12 ? i + 1 : 11] >> 3) != pos;
        const bool nf = feasible(state);
        const bool change = valid && last && nf != cur;
        const bool close = change && !nf;
        if (close && n < kMaxArcRanges) out[n] = (uint32_t)start | ((uint32_t)(pos - start) << 16);
        total += close ? pos - start : 0;
        n += close ? 1 : 0;
        start = (change && nf) ? pos : start;
        cur = change ? nf : cur;
    }
    if (cur) {
        if (n < kMaxArcRanges) out[n] = (uint32_t)start | ((uint32_t)(H - start) << 16);
        ++n;
        total += H - start;
    }
    if (n > kMaxArcRanges) {  // unusual: cover the whole radius instead
        out[0] = (uint32_t)H << 16;
        n = 1;
        total = H;
    }
    return n;
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
__device__ __forceinline__ Intervals intervals32(const TargetF32 T, const ChainF32 C, float2 r2,
                                              float4 sc, float half_w, int32_t clip) {
    const PairsT P = make_pairs(T);
    const PairsC PC = make_pairs(C);
    int yp[3], ym[3];
    float2 d[3];
    codes32<FAST, true>(P, PC, __fmul2_rn(r2, f2(sc.x, sc.y)), __fmul2_rn(r2, f2(sc.z, sc.w)),
                        half_w, yp, ym, d);
    Intervals I;
    I.any_flag = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int q = (s ? ym[c] : yp[c]) - kMagicBits;
            const float dd = s ? d[c].y : d[c].x;
            const bool f = fabsf(dd) >= half_w;
            I.any_flag |= f;
            const int j = 3 * s + c;
            I.lo[j] = q - ((f && dd < 0.0f) ? 1 : 0);
            I.hi[j] = q + ((f && dd >= 0.0f) ? 1 : 0);
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

// The luminance limit on an emitted pair (codes in [0, 255]): each colour's
// L* (step 1 applied to its codes, from the table of all 2^24 colours) lies
// within max_dl of the target's L*.
__device__ __forceinline__ bool dl_ok(const double* __restrict__ ltab, double max_dl,
                                      double l_target, const int qp[3], const int qm[3]) {
    const int ip = (qp[0] << 16) | (qp[1] << 8) | qp[2];
    const int im = (qm[0] << 16) | (qm[1] << 8) | qm[2];
    return fabs(__dsub_rn(__ldg(ltab + ip), l_target)) <= max_dl &&
           fabs(__dsub_rn(__ldg(ltab + im), l_target)) <= max_dl;
}

template <bool FAST>
__device__ __forceinline__ int certain32(const TargetF32& T, const ChainF32& C, float2 r2,
                                         float4 sc, float half_w, int32_t hi_min, int32_t lo_max,
                                         uint32_t mask2, int32_t clip, int list_mode) {
    const Intervals I = intervals32<FAST>(T, C, r2, sc, half_w, clip);
    return certain_from(I, hi_min, lo_max, mask2, clip, list_mode);
}


// ------------------------------------------------------------ angle-range items
// k_arc_ranges writes, per (target, radius) of a chunk, up to two slot ranges
// (start | len << 16; a third or more merged into the second, a superset),
// with bit 31 of the first word (kSlowRadius) set on a slow-path radius, whose
// slots the search evaluates with the slow chain.
// The search kernels concatenate, per warp, the ranges of up to kArcRadii
// radii into a list and evaluate only the listed slots, 32 at a time whatever
// radius they belong to; the rest certainly fail (k_search in increasing
// radius order, k_search_multi in decreasing radius rank).  List entry j:
// al[j] = radius offset (bits 0..6) | (first slot - first position +
// kArcBias) << 8, and its first position pos[j] =
// al[kArcEntries + j].  k_search lists the fast-path radii's entries first and
// the slow-path radii's after them, so that each region is walked by one chain
// variant; the first slow entry's position ends the fast region and a sentinel
// position ends the list.  After the list, al holds the start mask of the
// segment being walked (list_mask).
constexpr int kArcRadii = 128;
constexpr int kArcEntries = 2 * kArcRadii + 2;
constexpr int kArcMaskWords = 256;  // steps of 32 positions per segment, at most
constexpr int kArcWords = 2 * kArcEntries + kArcMaskWords;
constexpr int kArcBias = 1 << 23;
constexpr uint32_t kSlowRadius = 1u << 31;

__device__ __forceinline__ int warp_exclusive_sum(int v, int& total) {
    const unsigned lane = lane_id();
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if ((int)lane >= off) x += y;
    }
    total = __shfl_sync(0xFFFFFFFFu, x, 31);
    return x - v;
}

// The start mask of the positions [seg, seg + 32 nsteps) of a list region
// (entries below jend; nsteps <= kArcMaskWords), at al + 2 kArcEntries: bit l
// of word q is set where an entry starts at position seg + 32 q + l.  j0 is
// the entry holding position seg - 1 (jbeg - 1 before the region), so the
// entries from j0 + 1 on start at or after seg, in order.
__device__ __forceinline__ void list_mask(uint32_t* al, int jend, int seg, int nsteps, int j0) {
    const unsigned lane = lane_id();
    const uint32_t* pos = al + kArcEntries;
    uint32_t* msk = al + 2 * kArcEntries;
    for (int q = (int)lane; q < nsteps; q += 32) msk[q] = 0u;
    __syncwarp();
    const int end = seg + 32 * nsteps;
    for (int j = j0 + 1 + (int)lane;; j += 32) {
        const int pj = j < jend ? (int)pos[j] : end;
        const bool in = pj < end;
        if (in) atomicOr(msk + ((pj - seg) >> 5), 1u << ((pj - seg) & 31));
        if (!(__ballot_sync(0xFFFFFFFFu, in) >> 31)) break;  // later entries start later
    }
    __syncwarp();
}

// The slot of position b + lane of a list region, given `starts`, word
// (b - seg) / 32 of the segment's start mask: j0 is the entry holding position
// b - 1, and a lane's entry is j0 plus the starts at or before it.  Returns the
// entry word and advances j0 to the entry holding b + 31.
__device__ __forceinline__ uint32_t list_step(const uint32_t* al, uint32_t starts, int& j0) {
    const unsigned lane = lane_id();
    const int jj = j0 + __popc(starts & ((2u << lane) - 1u));
    j0 += __popc(starts);
    return al[jj];
}

// The entry of a list region [jbeg, jend) holding position p (the last one
// starting at or before p), by bisection over the start positions.
__device__ __forceinline__ uint32_t list_entry(const uint32_t* al, int jbeg, int jend, int p) {
    const uint32_t* pos = al + kArcEntries;
    int lo = jbeg, hi = jend - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int)pos[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return al[lo];
}

}  // namespace
}  // namespace cvs
