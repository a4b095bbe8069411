/*
 * cvs_oracle.c - plain, slow FP64 reference of the colour-pair search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing but tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header or table generator with the CUDA library.
 *
 * It follows the paper's §2 Methods step by step, as a serial loop over
 * target x radius i x angle j (the "simple serial loop" the paper attributes
 * to the prior method, §1 Introduction):
 *   1. decompose the target colour into L*, a*, b*            (§2, Fig. 2)
 *   2. add D_a = i sin j to a*, D_b = i cos j to b*; subtract for the
 *      point-symmetric partner; L* is kept fixed                 (§2, Fig. 1b)
 *   3. convert both colours back to 8-bit RGB
 *   4. keep the pairs that satisfy the embedding-signal condition: per RGB
 *      channel the pair's difference is "high" if it exceeds V_th and "low" if
 *      it is below V_th * R_novib (§3 Experiments, Table 1); the 3-bit
 *      high/low word is the embedded information (Table 1, patterns 100..111).
 * The colour-vibration (imperceptibility) condition is met by construction:
 * fixed L* and point symmetry about the target (§2 Methods).
 *
 * Readings where the paper is silent (constants, rounding, gamut): sRGB
 * IEC 61966-2-1 with D65 white; 8-bit code = floor(255*enc(lin) + 1/2) in exact
 * arithmetic, evaluated by counting quantisation thresholds; out-of-gamut
 * colours are rejected (gamut_mode 0) or clamped (gamut_mode 1).  All tables
 * arrive from the oracle's Python side (oracle/constants.py, oracle/trig.py).
 *
 * Build with -ffp-contract=off: every + - * / below is one IEEE operation in
 * the order written.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double M[3][3];   /* linear RGB -> XYZ */
    double W[3];      /* white point (Xn, Yn, Zn) */
    double MI[3][3];  /* XYZ -> linear RGB */
    double lut[256];  /* 8-bit sRGB decode */
    double thr[257];  /* quantisation thresholds, code k+1 starts at thr[k+1] */
    double f_break, finv_break, f_lin_mul, f_lin_add, finv_lin_mul;
} orc_consts;

typedef struct {
    uint16_t k, m;
    uint8_t plus[3], minus[3], pattern, flags;
    uint32_t target;
} orc_pair;

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ cbrt */
/* 192-bit unsigned integer, w[0] least significant. */
typedef struct { uint64_t w[3]; } u192;

static u192 cube_u54(uint64_t x) {           /* x < 2^54, returns x^3 */
    u128 sq = (u128)x * x;                    /* < 2^108 */
    u128 lo = (u128)(uint64_t)sq * x;         /* low 64 bits of sq times x */
    u128 hi = (u128)(uint64_t)(sq >> 64) * x; /* high part of sq times x */
    u192 r;
    r.w[0] = (uint64_t)lo;
    u128 mid = (lo >> 64) + (uint64_t)hi;
    r.w[1] = (uint64_t)mid;
    r.w[2] = (uint64_t)(hi >> 64) + (uint64_t)(mid >> 64);
    return r;
}

static u192 shl_u53(uint64_t x, int s) {      /* x * 2^s, 0 <= s < 139 */
    u192 r = {{0, 0, 0}};
    int limb = s / 64, bit = s % 64;
    u128 v = (u128)x << bit;                  /* x < 2^53, bit < 64: fits */
    if (limb < 3) r.w[limb] = (uint64_t)v;
    if (limb + 1 < 3) r.w[limb + 1] = (uint64_t)(v >> 64);
    return r;
}

static int cmp_u192(u192 a, u192 b) {
    for (int i = 2; i >= 0; --i) {
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    }
    return 0;
}

/* sign of (midpoint between z and its successor)^3 - t, for normal z, t > 0 */
static int mid_cube_vs(double z, double t) {
    int ez, et;
    double fz = frexp(z, &ez), ft = frexp(t, &et);
    uint64_t Z = (uint64_t)ldexp(fz, 53);     /* z = Z * 2^(ez-53) */
    uint64_t T = (uint64_t)ldexp(ft, 53);     /* t = T * 2^(et-53) */
    /* mid = (2Z+1) * 2^(ez-54); mid^3 = (2Z+1)^3 * 2^(3ez-162) */
    int sh = (et - 53) - (3 * ez - 162);      /* compare (2Z+1)^3 with T * 2^sh */
    u192 lhs = cube_u54(2 * Z + 1);
    if (sh < 0 || sh >= 139) {
        /* cannot happen for z within a few ulps of cbrt(t); decide by magnitude */
        return sh < 0 ? 1 : -1;
    }
    return cmp_u192(lhs, shl_u53(T, sh));
}

/* Correctly rounded cube root of a positive normal double. */
double orc_cbrt_cr(double t) {
    double y = cbrt(t);
    for (int it = 0; it < 8; ++it) {
        if (mid_cube_vs(y, t) < 0) {            /* t above the upper midpoint */
            y = nextafter(y, INFINITY);
            continue;
        }
        double ym = nextafter(y, 0.0);
        if (mid_cube_vs(ym, t) > 0) {           /* t below the lower midpoint */
            y = ym;
            continue;
        }
        break;
    }
    return y;
}

/* ------------------------------------------------------------------ colour */
static double cie_f(const orc_consts* C, double t) {
    if (t > C->f_break) return orc_cbrt_cr(t);
    return t * C->f_lin_mul + C->f_lin_add;
}

static double cie_finv(const orc_consts* C, double u) {
    if (u > C->finv_break) return (u * u) * u;
    return (u - C->f_lin_add) * C->finv_lin_mul;
}

/* Linear RGB -> L*, a*, b* (CIE 1976, white W). */
void orc_lin_to_lab(const orc_consts* C, const double lin[3], double lab[3]) {
    double xyz[3];
    for (int i = 0; i < 3; ++i)
        xyz[i] = (C->M[i][0] * lin[0] + C->M[i][1] * lin[1]) + C->M[i][2] * lin[2];
    double fx = cie_f(C, xyz[0] / C->W[0]);
    double fy = cie_f(C, xyz[1] / C->W[1]);
    double fz = cie_f(C, xyz[2] / C->W[2]);
    lab[0] = 116.0 * fy - 16.0;
    lab[1] = 500.0 * (fx - fy);
    lab[2] = 200.0 * (fy - fz);
}

/* Step 1: 8-bit sRGB target -> L*, a*, b* (decode through the table). */
void orc_target_lab(const orc_consts* C, const uint8_t rgb[3], double lab[3]) {
    double lin[3] = {C->lut[rgb[0]], C->lut[rgb[1]], C->lut[rgb[2]]};
    orc_lin_to_lab(C, lin, lab);
}

/* Step 1 for many targets: rgb (3n bytes) -> lab (3n doubles). */
void orc_target_lab_many(const orc_consts* C, const uint8_t* rgb, int64_t n, double* lab,
                         int n_threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads)
#endif
    for (int64_t t = 0; t < n; ++t) orc_target_lab(C, rgb + 3 * t, lab + 3 * t);
    (void)n_threads;
}

/* Step 3a: L*, a*, b* -> linear RGB. */
void orc_lab_to_lin(const orc_consts* C, double L, double a, double b, double lin[3]) {
    double fy = (L + 16.0) / 116.0;
    double fx = fy + a / 500.0;
    double fz = fy - b / 200.0;
    double X = C->W[0] * cie_finv(C, fx);
    double Y = C->W[1] * cie_finv(C, fy);
    double Z = C->W[2] * cie_finv(C, fz);
    for (int c = 0; c < 3; ++c)
        lin[c] = (C->MI[c][0] * X + C->MI[c][1] * Y) + C->MI[c][2] * Z;
}

/* Step 3b: linear value -> 8-bit code, floor(255 enc(lin) + 1/2) clamped to
 * [-1, 256]: the number of thresholds not above lin, minus one. */
int orc_quantize(const orc_consts* C, double lin) {
    int lo = 0, hi = 257;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (C->thr[mid] <= lin) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

/* The same code from the textbook formula with libm pow (for cross-checks
 * only; it can differ from orc_quantize only within rounding of a tie). */
int orc_quantize_pow(double lin) {
    double e = lin <= 0.0031308 ? 12.92 * lin : 1.055 * pow(lin, 1.0 / 2.4) - 0.055;
    double q = floor(255.0 * e + 0.5);
    if (q < -1.0) q = -1.0;
    if (q > 256.0) q = 256.0;
    return (int)q;
}

/* Step 4: per channel, 1 = high (diff > V_th), 0 = low (diff < V_th*R_novib,
 * compared exactly through one fused multiply-add), -1 = neither. */
static int classify(int diff, double v_th, double r_novib) {
    double d = (double)diff;
    if (d > v_th) return 1;
    if (fma(v_th, r_novib, -d) > 0.0) return 0;
    return -1;
}

/* Decide one point-symmetric pair.  q_plus / q_minus are the raw codes in
 * [-1, 256].  Returns the pattern (1..7) if the pair passes, else 0. The codes
 * as emitted (after clamping in clip mode) are written to out_plus/out_minus. */
static int decide_pair(const int q_plus[3], const int q_minus[3], double v_th, double r_novib,
                       uint32_t pattern_mask, int gamut_mode, uint8_t out_plus[3],
                       uint8_t out_minus[3]) {
    int p[3], m[3];
    for (int c = 0; c < 3; ++c) {
        p[c] = q_plus[c];
        m[c] = q_minus[c];
        if (gamut_mode == 1) {
            if (p[c] < 0) p[c] = 0;
            if (p[c] > 255) p[c] = 255;
            if (m[c] < 0) m[c] = 0;
            if (m[c] > 255) m[c] = 255;
        } else if (p[c] < 0 || p[c] > 255 || m[c] < 0 || m[c] > 255) {
            return 0;
        }
    }
    int pattern = 0;
    for (int c = 0; c < 3; ++c) {
        int diff = p[c] > m[c] ? p[c] - m[c] : m[c] - p[c];
        int cls = classify(diff, v_th, r_novib);
        if (cls < 0) return 0;
        pattern |= cls << (2 - c);   /* R is the leading digit, as in Table 1 */
    }
    if (pattern == 0) return 0;
    if (!((pattern_mask >> (pattern - 1)) & 1u)) return 0;
    for (int c = 0; c < 3; ++c) {
        out_plus[c] = (uint8_t)p[c];
        out_minus[c] = (uint8_t)m[c];
    }
    return pattern;
}

/* Perceptual refinement of the vibration condition (a reading: the paper fixes
 * L* before quantisation, §2 Methods, and gives no tolerance after it): each
 * emitted 8-bit colour's L* (step 1 applied to its codes) must lie within
 * max_dl of the target's L*.  max_dl < 0 or NaN: no limit. */
static int passes_dl(const orc_consts* C, double L_target, const uint8_t op[3],
                     const uint8_t om[3], double max_dl) {
    if (!(max_dl >= 0.0)) return 1;
    double lp[3], lm[3];
    orc_target_lab(C, op, lp);
    orc_target_lab(C, om, lm);
    return fabs(lp[0] - L_target) <= max_dl && fabs(lm[0] - L_target) <= max_dl;
}

/* Exported form of passes_dl for the oracle's own pins. */
int orc_passes_dl(const orc_consts* C, double L_target, const uint8_t op[3], const uint8_t om[3],
                  double max_dl) {
    return passes_dl(C, L_target, op, om, max_dl);
}

/* Exported form of decide_pair for the oracle's own pins. */
int orc_decide_pair(const int q_plus[3], const int q_minus[3], double v_th, double r_novib,
                    uint32_t pattern_mask, int gamut_mode, uint8_t out_plus[3],
                    uint8_t out_minus[3]) {
    return decide_pair(q_plus, q_minus, v_th, r_novib, pattern_mask, gamut_mode, out_plus,
                       out_minus);
}

/* Both colours of candidate (radius r, table entries s = sin j, c = cos j). */
void orc_pair_codes(const orc_consts* C, const double lab[3], double r, double s, double c,
                    int q_plus[3], int q_minus[3]) {
    double da = r * s, db = r * c;           /* D_a, D_b entries */
    double lin[3];
    orc_lab_to_lin(C, lab[0], lab[1] + da, lab[2] + db, lin);
    for (int ch = 0; ch < 3; ++ch) q_plus[ch] = orc_quantize(C, lin[ch]);
    orc_lab_to_lin(C, lab[0], lab[1] - da, lab[2] - db, lin);
    for (int ch = 0; ch < 3; ++ch) q_minus[ch] = orc_quantize(C, lin[ch]);
}

/* One target colour: every passing (k, m) in (k, m) order, up to cap records.
 * Returns the total number of passing candidates (which may exceed cap). */
int64_t orc_search_color(const orc_consts* C, const uint8_t rgb[3], uint32_t target,
                         const double* radii, int32_t n_radii, const double* sin_t,
                         const double* cos_t, int32_t n_angles, double v_th, double r_novib,
                         uint32_t pattern_mask, int gamut_mode, double max_dl, orc_pair* out,
                         int64_t cap) {
    double lab[3];
    orc_target_lab(C, rgb, lab);
    int64_t n = 0;
    for (int32_t k = 0; k < n_radii; ++k) {
        for (int32_t m = 0; m < n_angles; ++m) {
            int qp[3], qm[3];
            orc_pair_codes(C, lab, radii[k], sin_t[m], cos_t[m], qp, qm);
            orc_pair rec;
            memset(&rec, 0, sizeof rec);
            int pat = decide_pair(qp, qm, v_th, r_novib, pattern_mask, gamut_mode, rec.plus,
                                  rec.minus);
            if (!pat || !passes_dl(C, lab[0], rec.plus, rec.minus, max_dl)) continue;
            if (n < cap) {
                rec.k = (uint16_t)k;
                rec.m = (uint16_t)m;
                rec.pattern = (uint8_t)pat;
                rec.target = target;
                out[n] = rec;
            }
            ++n;
        }
    }
    return n;
}

/* Many targets: per target the number of passing (k, m), the largest passing
 * radius (-1 if none) and the set of passing patterns (bit p-1 for pattern p). */
void orc_search_colors(const orc_consts* C, const uint8_t* rgb, int64_t n_targets,
                       const double* radii, int32_t n_radii, const double* sin_t,
                       const double* cos_t, int32_t n_angles, double v_th, double r_novib,
                       uint32_t pattern_mask, int gamut_mode, double max_dl, float* max_r,
                       int32_t* count, uint8_t* pmask, int n_threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t t = 0; t < n_targets; ++t) {
        double lab[3];
        orc_target_lab(C, rgb + 3 * t, lab);
        int32_t cnt = 0;
        double best = -1.0;
        uint8_t mask = 0;
        for (int32_t k = 0; k < n_radii; ++k) {
            for (int32_t m = 0; m < n_angles; ++m) {
                int qp[3], qm[3];
                uint8_t op[3], om[3];
                orc_pair_codes(C, lab, radii[k], sin_t[m], cos_t[m], qp, qm);
                int pat = decide_pair(qp, qm, v_th, r_novib, pattern_mask, gamut_mode, op, om);
                if (!pat || !passes_dl(C, lab[0], op, om, max_dl)) continue;
                ++cnt;
                if (radii[k] > best) best = radii[k];
                mask |= (uint8_t)(1u << (pat - 1));
            }
        }
        count[t] = cnt;
        max_r[t] = (float)best;
        pmask[t] = mask;
    }
    (void)n_threads;
}

/* Embedding (Fig. 1a: devices see an area that looks uniform to people switch
 * between two colours).  Per pixel i with requested pattern p = pattern[i] in
 * 1..7: among the candidates (k, m) whose pair passes with exactly pattern p
 * (and, with a luminance limit max_dl >= 0, passes it too), take the first in
 * (radius value, k, m) order - the smallest colour shift, then the caller's
 * radius and angle order.  Frame A gets the pair's "plus" colour (a* + D_a,
 * b* + D_b), frame B its "minus" colour.  Pixels with p outside 1..7, or with
 * no such candidate, keep their own colour in both frames.  choice[i] =
 * k | m << 16, or 0xFFFFFFFF when nothing was embedded.  rgb, frame_a,
 * frame_b: 3 bytes per pixel, dense. */
void orc_embed(const orc_consts* C, const uint8_t* rgb, const uint8_t* pattern,
               int64_t n_pixels, const double* radii, int32_t n_radii, const double* sin_t,
               const double* cos_t, int32_t n_angles, double v_th, double r_novib,
               uint32_t pattern_mask, int gamut_mode, double max_dl, uint8_t* frame_a,
               uint8_t* frame_b, uint32_t* choice, int n_threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t i = 0; i < n_pixels; ++i) {
        const uint8_t* src = rgb + 3 * i;
        int p = pattern[i];
        int found = 0;
        double best_r = 0.0;
        uint32_t best = 0xFFFFFFFFu;
        uint8_t best_plus[3] = {src[0], src[1], src[2]};
        uint8_t best_minus[3] = {src[0], src[1], src[2]};
        if (p >= 1 && p <= 7) {
            double lab[3];
            orc_target_lab(C, src, lab);
            for (int32_t k = 0; k < n_radii; ++k) {
                /* (k, m) run in increasing order, so only a strictly smaller
                 * radius value can replace an earlier candidate */
                if (found && !(radii[k] < best_r)) continue;
                for (int32_t m = 0; m < n_angles; ++m) {
                    int qp[3], qm[3];
                    uint8_t op[3], om[3];
                    orc_pair_codes(C, lab, radii[k], sin_t[m], cos_t[m], qp, qm);
                    if (decide_pair(qp, qm, v_th, r_novib, pattern_mask, gamut_mode, op, om) != p ||
                        !passes_dl(C, lab[0], op, om, max_dl))
                        continue;
                    found = 1;
                    best_r = radii[k];
                    best = (uint32_t)k | ((uint32_t)m << 16);
                    memcpy(best_plus, op, 3);
                    memcpy(best_minus, om, 3);
                    break;  /* the smallest m of this radius */
                }
            }
        }
        memcpy(frame_a + 3 * i, best_plus, 3);
        memcpy(frame_b + 3 * i, best_minus, 3);
        choice[i] = best;
    }
    (void)n_threads;
}

/* Self-check over all 2^24 8-bit colours: RGB -> Lab -> linear RGB must give
 * back the decode table within max_err, and the same 8-bit codes.  Returns the
 * number of colours whose codes differ; *max_err receives the largest
 * |lin - LUT| seen. */
int64_t orc_roundtrip_all(const orc_consts* C, double* max_err, int n_threads) {
    int64_t bad = 0;
    double worst = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads) reduction(+:bad) reduction(max:worst)
#endif
    for (int64_t v = 0; v < (1 << 24); ++v) {
        uint8_t rgb[3] = {(uint8_t)(v >> 16), (uint8_t)(v >> 8), (uint8_t)v};
        double lab[3], lin[3];
        orc_target_lab(C, rgb, lab);
        orc_lab_to_lin(C, lab[0], lab[1], lab[2], lin);
        for (int c = 0; c < 3; ++c) {
            double e = fabs(lin[c] - C->lut[rgb[c]]);
            if (e > worst) worst = e;
            if (orc_quantize(C, lin[c]) != rgb[c]) { ++bad; break; }
        }
    }
    *max_err = worst;
    (void)n_threads;
    return bad;
}

int orc_openmp_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
