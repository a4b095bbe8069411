// cvs_device.cuh - device arithmetic of libcvsearch (sm_103a).
//
// Paper: §2 Methods (target -> L*a*b*, D_a = i sin j, D_b = i cos j added to /
// subtracted from a*, b* at fixed L*, back to RGB), §3 Experiments and Table 1
// (embedding-signal condition with V_th, R_novib; patterns 100..111).
//
// Two evaluations of one candidate colour exist:
//   * FP64, in the exact operation order of the textbook formulas, every
//     operation an explicit IEEE intrinsic (no contraction).  This defines the
//     result and is what the FP64 comparison path and the re-decision use.
//   * FP32, relative to the target: the cube (f^-1) is expanded around the
//     target's f-values, so only the small displacement is rounded at FP32
//     precision; the sRGB encode uses MUFU lg2/ex2.  A code whose unrounded
//     value lies within the window W of a rounding boundary is "flagged" and
//     re-decided in FP64 when the flag could change the result.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cvs_tables.h"

namespace cvs {

// ----------------------------------------------------------------- constants
__constant__ double c_M[9] = CVS_M_INIT;
__constant__ double c_W[3] = CVS_W_INIT;
__constant__ double c_MI[9] = CVS_MI_INIT;
__constant__ double c_sin_c[2 * CVS_N_SIN_C] = CVS_SIN_C_INIT;
__constant__ double c_cos_c[2 * CVS_N_COS_C] = CVS_COS_C_INIT;
// Tables indexed per lane (divergent): global memory, read through L1.
__device__ const double g_decode[256] = CVS_DECODE_INIT;
__device__ const double g_qthr[257] = CVS_QTHR_INIT;

constexpr double kFBreak = CVS_F_BREAK;
constexpr double kFinvBreak = CVS_FINV_BREAK;
constexpr double kFLinMul = CVS_F_LIN_MUL;
constexpr double kFLinAdd = CVS_F_LIN_ADD;
constexpr double kFinvLinMul = CVS_FINV_LIN_MUL;

// 1.5 * 2^23: v + kMagic rounds v to an integer held in the low mantissa bits.
constexpr float kMagic = 12582912.0f;
constexpr int32_t kMagicBits = 0x4B400000;

// ----------------------------------------------------------- per-target data
// FP32 constants of one target for the relative chain (48 bytes).
//   c1x = 3 fx0, c2x = 3 fx0^2: (fx0+u)^3 - fx0^3 = u (c2x + u (c1x + u))
//   fx0, fz0: f-values of the target (as the FP64 inverse chain forms them)
//   X30, Z30: f^-1(fx0), f^-1(fz0) (slow path, which handles the linear branch)
//   lin0[3]: linear RGB of the target as the FP64 inverse chain produces it
//   flags: bit 0 = every candidate stays on the cubic branch (fast path)
struct __align__(16) TargetF32 {
    float c1x, c2x, c1z, c2z;
    float fx0, fz0, X30, Z30;
    float lin0[3];
    uint32_t flags;
};

// FP64 L*a*b* of one target plus where its results go (32 bytes).
struct __align__(16) TargetF64 {
    double L, a, b;
    uint64_t out_slot;  // colours: index; images: (image << 40) | pixel
};

// Shared FP32 matrix columns: lin_c += Ax[c] * dX3 + Bz[c] * dZ3.
struct ChainF32 {
    float Ax[3], Bz[3];
};

// ----------------------------------------------------- correctly rounded cbrt
// Sign of m^3 - t, where m is the midpoint between z and the next double up
// (z, t positive normal doubles).  Exact: 192-bit integer arithmetic.
__device__ __forceinline__ int mid_cube_sign(double z, double t) {
    const uint64_t zb = (uint64_t)__double_as_longlong(z);
    const uint64_t tb = (uint64_t)__double_as_longlong(t);
    const int ez = (int)(zb >> 52) - 1075;  // z = Zm * 2^ez, Zm with hidden bit
    const int et = (int)(tb >> 52) - 1075;
    const uint64_t Zm = (zb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const uint64_t Tm = (tb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    // m = (2 Zm + 1) 2^(ez-1);  m^3 = C 2^(3ez-3) with C = (2 Zm + 1)^3 < 2^162
    const uint64_t o = 2 * Zm + 1;
    const uint64_t sq_lo = o * o, sq_hi = __umul64hi(o, o);
    const uint64_t a0 = sq_lo * o, a1 = __umul64hi(sq_lo, o);
    const uint64_t b0 = sq_hi * o, b1 = __umul64hi(sq_hi, o);
    const uint64_t c0 = a0;
    const uint64_t c1 = a1 + b0;
    const uint64_t c2 = b1 + (c1 < a1 ? 1ull : 0ull);
    // t = Tm 2^et; compare C with Tm 2^s, s = et - 3ez + 3
    const int s = et - 3 * ez + 3;
    if (s < 0) return 1;     // t tiny against m^3 (not reached for z ~ cbrt(t))
    if (s > 138) return -1;  // t huge against m^3 (not reached)
    uint64_t d0 = 0, d1 = 0, d2 = 0;
    const int limb = s >> 6, bit = s & 63;
    const uint64_t lo = Tm << bit;
    const uint64_t hi = bit ? (Tm >> (64 - bit)) : 0ull;
    if (limb == 0) { d0 = lo; d1 = hi; }
    else if (limb == 1) { d1 = lo; d2 = hi; }
    else { d2 = lo; }
    if (c2 != d2) return c2 < d2 ? -1 : 1;
    if (c1 != d1) return c1 < d1 ? -1 : 1;
    if (c0 != d0) return c0 < d0 ? -1 : 1;
    return 0;  // impossible: the cube of an odd 54-bit number has > 53 bits
}

// Cube root of a positive normal double, correctly rounded to nearest.
static __device__ __noinline__ double cbrt_rn(double t) {
    double y = cbrt(t);  // within a few ulps
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        if (mid_cube_sign(y, t) < 0) { y = nextafter(y, 2.0); continue; }
        const double ylo = nextafter(y, 0.0);
        if (mid_cube_sign(ylo, t) > 0) { y = ylo; continue; }
        break;
    }
    return y;
}

// ------------------------------------------------------------ FP64 chain
__device__ __forceinline__ double cie_f64(double t) {
    return t > kFBreak ? cbrt_rn(t) : __dadd_rn(__dmul_rn(t, kFLinMul), kFLinAdd);
}

__device__ __forceinline__ double cie_finv64(double u) {
    return u > kFinvBreak ? __dmul_rn(__dmul_rn(u, u), u)
                          : __dmul_rn(__dsub_rn(u, kFLinAdd), kFinvLinMul);
}

// Step 1 of §2 Methods: 8-bit sRGB -> L*, a*, b* (FP64, textbook order).
__device__ __forceinline__ void target_lab64(uint32_t r8, uint32_t g8, uint32_t b8, double& L,
                                             double& a, double& b) {
    const double lin0 = g_decode[r8], lin1 = g_decode[g8], lin2 = g_decode[b8];
    double xyz[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        xyz[i] = __dadd_rn(__dadd_rn(__dmul_rn(c_M[3 * i], lin0), __dmul_rn(c_M[3 * i + 1], lin1)),
                           __dmul_rn(c_M[3 * i + 2], lin2));
    }
    const double fx = cie_f64(__ddiv_rn(xyz[0], c_W[0]));
    const double fy = cie_f64(__ddiv_rn(xyz[1], c_W[1]));
    const double fz = cie_f64(__ddiv_rn(xyz[2], c_W[2]));
    L = __dsub_rn(__dmul_rn(116.0, fy), 16.0);
    a = __dmul_rn(500.0, __dsub_rn(fx, fy));
    b = __dmul_rn(200.0, __dsub_rn(fy, fz));
}

// Monotone integer key of a double (for exact comparisons on the integer pipe).
__device__ __forceinline__ long long dkey(double x) {
    long long k = __double_as_longlong(x);
    return k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// Forward declaration: FP32 encode used as the starting guess.
__device__ __forceinline__ float encode_v32(float lin);

// floor(255 enc(lin) + 1/2) of a double in exact arithmetic, clamped to [-1,256]:
// the number of quantisation thresholds not above lin, minus one.
__device__ __forceinline__ int quantize64(double lin, const long long* __restrict__ qkey) {
    const float v = encode_v32((float)lin);
    int q = (int)fminf(fmaxf(rintf(v), -1.0f), 256.0f);
    const long long k = dkey(lin);
#pragma unroll 1
    while (q < 256 && __ldg(qkey + q + 1) <= k) ++q;
#pragma unroll 1
    while (q >= 0 && k < __ldg(qkey + q)) --q;
    return q;
}

// Step 3 of §2 Methods in FP64 for one colour (L, a + da, b + db): codes.
__device__ __forceinline__ void color_codes64(double L, double a2, double b2,
                                              const long long* __restrict__ qkey, int q[3]) {
    const double fy = __ddiv_rn(__dadd_rn(L, 16.0), 116.0);
    const double fx = __dadd_rn(fy, __ddiv_rn(a2, 500.0));
    const double fz = __dsub_rn(fy, __ddiv_rn(b2, 200.0));
    const double X = __dmul_rn(c_W[0], cie_finv64(fx));
    const double Y = __dmul_rn(c_W[1], cie_finv64(fy));
    const double Z = __dmul_rn(c_W[2], cie_finv64(fz));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double lin = __dadd_rn(__dadd_rn(__dmul_rn(c_MI[3 * c], X), __dmul_rn(c_MI[3 * c + 1], Y)),
                                     __dmul_rn(c_MI[3 * c + 2], Z));
        q[c] = quantize64(lin, qkey);
    }
}

// Linear RGB of one colour in FP64 (same chain, before quantisation).
__device__ __forceinline__ void color_lin64(double L, double a2, double b2, double lin[3]) {
    const double fy = __ddiv_rn(__dadd_rn(L, 16.0), 116.0);
    const double fx = __dadd_rn(fy, __ddiv_rn(a2, 500.0));
    const double fz = __dsub_rn(fy, __ddiv_rn(b2, 200.0));
    const double X = __dmul_rn(c_W[0], cie_finv64(fx));
    const double Y = __dmul_rn(c_W[1], cie_finv64(fy));
    const double Z = __dmul_rn(c_W[2], cie_finv64(fz));
#pragma unroll
    for (int c = 0; c < 3; ++c)
        lin[c] = __dadd_rn(__dadd_rn(__dmul_rn(c_MI[3 * c], X), __dmul_rn(c_MI[3 * c + 1], Y)),
                           __dmul_rn(c_MI[3 * c + 2], Z));
}

// Both colours of candidate (r, sin j, cos j) for a target: D_a = r sin j and
// D_b = r cos j added (plus) and subtracted (minus), L* fixed.
__device__ __forceinline__ void pair_codes64(double L, double a, double b, double r, double s,
                                             double c, const long long* __restrict__ qkey,
                                             int qp[3], int qm[3]) {
    const double da = __dmul_rn(r, s), db = __dmul_rn(r, c);
    color_codes64(L, __dadd_rn(a, da), __dadd_rn(b, db), qkey, qp);
    color_codes64(L, __dsub_rn(a, da), __dsub_rn(b, db), qkey, qm);
}

// ------------------------------------------------------- decision (integers)
// Embedding-signal condition (§3 Experiments, Table 1) on the 8-bit codes.
struct Decide {
    int32_t hi_min;     // difference >= hi_min  <=>  high (> V_th)
    int32_t lo_max;     // difference <= lo_max  <=>  low  (< V_th * R_novib)
    uint32_t mask2;     // pattern mask shifted left by one: bit p enables pattern p
    int32_t clip;       // gamut mode 1
};

// Returns the pattern (1..7) if the pair passes, else 0.  Codes in [-1, 256].
__device__ __forceinline__ int decide_codes(const int qp_in[3], const int qm_in[3], const Decide& D) {
    int qp[3], qm[3];
    bool in_gamut = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        qp[c] = qp_in[c];
        qm[c] = qm_in[c];
        if (D.clip) {
            qp[c] = min(max(qp[c], 0), 255);
            qm[c] = min(max(qm[c], 0), 255);
        } else {
            in_gamut &= (unsigned)qp[c] <= 255u && (unsigned)qm[c] <= 255u;
        }
    }
    int pattern = 0;
    bool valid = in_gamut;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int d = abs(qp[c] - qm[c]);
        const bool hi = d >= D.hi_min;
        const bool lo = d <= D.lo_max;
        valid &= hi || lo;
        pattern |= (hi ? 1 : 0) << (2 - c);
    }
    valid &= ((D.mask2 >> pattern) & 1u) != 0u;  // bit 0 of mask2 is 0: pattern 000 fails
    return valid ? pattern : 0;
}

// ------------------------------------------------------------- FP32 encode
// v = 255 enc(lin) before rounding; sRGB encode with MUFU lg2 / ex2.
__device__ __forceinline__ float encode_v32(float lin) {
    float lg, p;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(lin));
    const float t = lg * (5.0f / 12.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p) : "f"(t));
    const float vpow = fmaf(269.025f, p, -14.025f);  // 255 (1.055 p - 0.055)
    const float vlin = lin * 3294.6f;                // 255 * 12.92 lin
    return lin <= 0.0031308f ? vlin : vpow;
}

// ------------------------------------------------------ double-double trig
struct dd_t { double hi, lo; };

__device__ __forceinline__ dd_t two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dd_t fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd_t dd_add(dd_t x, dd_t y) {
    dd_t s = two_sum(x.hi, y.hi);
    dd_t t = two_sum(x.lo, y.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd_t dd_mul(dd_t x, dd_t y) {
    const double p = __dmul_rn(x.hi, y.hi);
    double e = __fma_rn(x.hi, y.hi, -p);
    e = __fma_rn(x.hi, y.lo, e);
    e = __fma_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// sin and cos of x degrees for x in [0, 45], as double-double.
static __device__ void sincos_dd_deg(double x, dd_t& s, dd_t& c) {
    // t = x * pi/180 (double-double)
    const double p = __dmul_rn(x, CVS_PI180_HI);
    double e = __fma_rn(x, CVS_PI180_HI, -p);
    e = __fma_rn(x, CVS_PI180_LO, e);
    const dd_t t = fast_two_sum(p, e);
    const dd_t t2 = dd_mul(t, t);
    // Horner in t^2: sin = t (c0 + t2 (c1 + ...)), cos = 1 + t2 (d0 + t2 (d1 + ...))
    dd_t ss = {c_sin_c[2 * (CVS_N_SIN_C - 1)], c_sin_c[2 * (CVS_N_SIN_C - 1) + 1]};
    for (int i = CVS_N_SIN_C - 2; i >= 0; --i)
        ss = dd_add(dd_mul(ss, t2), dd_t{c_sin_c[2 * i], c_sin_c[2 * i + 1]});
    s = dd_mul(ss, t);
    dd_t cc = {c_cos_c[2 * (CVS_N_COS_C - 1)], c_cos_c[2 * (CVS_N_COS_C - 1) + 1]};
    for (int i = CVS_N_COS_C - 2; i >= 0; --i)
        cc = dd_add(dd_mul(cc, t2), dd_t{c_cos_c[2 * i], c_cos_c[2 * i + 1]});
    c = dd_add(dd_mul(cc, t2), dd_t{1.0, 0.0});
}

// Round a double-double to the nearest double; *uncertain is set if its
// accuracy (about 1e-30 relative) does not settle the rounding.
__device__ __forceinline__ double dd_round(dd_t v, int* uncertain) {
    const dd_t n = fast_two_sum(v.hi, v.lo);
    if (n.hi != 0.0 && n.lo != 0.0) {
        // half the gap to the neighbouring double on the side of the low word
        const double nb = nextafter(n.hi, n.lo > 0.0 ? 2.0 * n.hi : 0.0);
        const double half_gap = 0.5 * fabs(__dsub_rn(nb, n.hi));
        if (fabs(fabs(n.lo) - half_gap) < 1e-29 * fabs(n.hi)) *uncertain = 1;
    }
    return n.hi;
}

// Correctly rounded sin / cos of an angle in degrees (any finite double).
// The reduction to [0, 45] degrees is exact (fmod, then subtractions that
// Sterbenz's lemma makes exact), so sin(j + 180) = -sin(j) bit for bit.
static __device__ void sincos_deg_rn(double deg, double* s_out, double* c_out, int* uncertain) {
    const bool neg = deg < 0.0;
    double t = fmod(fabs(deg), 360.0);  // exact, in [0, 360)
    double ssign = 1.0, csign = 1.0;
    if (t > 270.0) { t = __dsub_rn(360.0, t); ssign = -1.0; }           // sin(360-t) = -sin t
    else if (t > 180.0) { t = __dsub_rn(t, 180.0); ssign = -1.0; csign = -1.0; }
    else if (t > 90.0) { t = __dsub_rn(180.0, t); csign = -1.0; }
    // now t in [0, 90]
    dd_t sd, cd;
    bool swap = false;
    if (t > 45.0) { t = __dsub_rn(90.0, t); swap = true; }
    if (t == 0.0) { sd = {0.0, 0.0}; cd = {1.0, 0.0}; }
    else sincos_dd_deg(t, sd, cd);
    double sv = dd_round(sd, uncertain), cv = dd_round(cd, uncertain);
    if (swap) { const double tmp = sv; sv = cv; cv = tmp; }
    sv *= ssign;
    cv *= csign;
    if (neg) sv = -sv;
    *s_out = sv + 0.0;  // +0.0 for zero results, never -0.0
    *c_out = cv + 0.0;
}

}  // namespace cvs
