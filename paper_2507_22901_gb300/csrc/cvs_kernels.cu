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
//             whose FP32 codes sit within W of a rounding boundary are marked
//             in a per-lane bitmap, decided after each segment by exact
//             interval analysis (32 at a time), and, where that cannot decide,
//             re-decided in FP64 (one slot per lane).
// The FP32 slot itself (chain, decision, interval analysis) is in
// cvs_slot32.cuh; the multi-threshold search is in cvs_multi.cu.
//   finalize: per-target accumulators -> caller's capacity maps.
// When the angle list is closed under +180 degrees, slot h covers angles h and
// h + N/2: the "minus" colour of one is the "plus" colour of the other.
#include <cuda_runtime.h>

#include "cvs_device.cuh"
#include "cvs_internal.h"
#include "cvs_slot32.cuh"

namespace cvs {

namespace {

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

// ------------------------------------------------------------ search kernel
struct Smem {
    float2* r2;     // K: (r, r)
    float4* sc4;    // H: (sin/500, -sin/500, -cos/200, cos/200)
    uint8_t* lut;   // 3 x 512 channel-difference classes
    uint32_t* rq_t; // per warp: kRqCap target indices (low 32 bits)
    uint32_t* rq_kh;
};

// Pair lists (list mode).  A work item (target t, radii [k0, k1)) marks its
// passing slots s = (k - k0) H + h in a per-warp bitmap in shared memory,
// wherever the slot is decided (the FP32 walk, the interval analysis of
// flagged slots, the FP64 re-decision); once every slot of the item is decided
// it writes its records, in (k, m) order, straight to their final place (see
// emit_item).
__device__ __forceinline__ void mark_pass(uint32_t* pb, int k0, int H, int k, int h) {
    const int s = (k - k0) * H + h;
    atomicOr(pb + (s >> 5), 1u << (s & 31));
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
    const int pattern = decide_codes(qp, qm, dc);
    return (pattern && A.ltab && !dl_ok(A.ltab, A.max_dl, D.L, qp, qm)) ? 0 : pattern;
}

// The warp's current work item in list mode: its bitmap in shared memory (pb,
// NULL when there is none), target and radii [k0, k1).
struct ItemRef {
    uint32_t* pb;
    int64_t t;
    int k0, k1;
};

// A passing slot of an earlier, already stored item (list mode): straight
// into that item's bitmap and count in global memory.
__device__ __forceinline__ void mark_stored(const SearchArgs& A, int64_t t, int k, int h) {
    const int kchunk = A.shape.kchunk;
    const int n_kc = (A.grid.K + kchunk - 1) / kchunk;
    const int kc = k / kchunk;
    const long long g = A.item0 + t * (long long)n_kc + kc;
    const int s = (k - kc * kchunk) * A.grid.H + h;
    atomicOr(A.item_bits + g * (long long)A.item_words + (s >> 5), 1u << (s & 31));
    atomicAdd(A.item_count + g, 1u);
}

// Re-decide up to 32 queued slots in FP64, one per lane, and merge them.  The
// queue runs across work items; in list mode a slot of the current item goes
// to its bitmap in shared memory, a slot of an earlier item to global memory.
__device__ __noinline__ void flush_queue(const SearchArgs& A, uint32_t* rq_t, uint32_t* rq_kh,
                                         int n, unsigned long long* n_re, uint32_t* cur_pb,
                                         int64_t cur_t, int cur_k0, int cur_k1) {
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
                if (cur_pb && (int64_t)t == cur_t && k >= cur_k0 && k < cur_k1)
                    mark_pass(cur_pb, cur_k0, A.grid.H, k, h);
                else
                    mark_stored(A, (int64_t)t, k, h);
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
                                          unsigned long long& n_re, const ItemRef& cur) {
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
        flush_queue(A, rq_t, rq_kh, 32, &n_re, cur.pb, cur.t, cur.k0, cur.k1);
        const int rest = rq_n - 32;
        uint32_t mt = 0, mkh = 0;
        if ((int)lane < rest) { mt = rq_t[32 + lane]; mkh = rq_kh[32 + lane]; }
        __syncwarp();
        if ((int)lane < rest) { rq_t[lane] = mt; rq_kh[lane] = mkh; }
        __syncwarp();
        rq_n = rest;
    }
}

// Per-lane accumulators of one work item, and in list mode its bitmap.
struct Tally {
    int cnt;
    float rmax;
    uint32_t pm;
    uint32_t skip;   // slots of this lane skipped as certainly out of gamut
    uint32_t prune;  // slots of the item below the first radius where a pair may pass
    ItemRef item;    // list mode: the current item (its bitmap in shared memory), else pb NULL
};

// Decide up to 32 flagged slots of target t, one per lane: exact interval
// analysis in FP32, FP64 re-decision where the analysis cannot decide.  A list
// takes the codes of a passing slot later (emit_item), so only the luminance
// limit needs them exactly here.
template <bool FAST, bool DL>
__device__ __forceinline__ void drain_flagged(const SearchArgs& A, const Smem& S,
                                              const TargetF32& T, const ChainF32& C, int64_t t,
                                              uint32_t* pq, int n, Tally& acc, uint32_t* rq_t,
                                              uint32_t* rq_kh, int& rq_n,
                                              unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int inc = A.grid.sym ? 2 : 1;
    int k = 0, h = 0, pc = 0;
    if ((int)lane < n) {
        const uint32_t kh = pq[lane];
        k = (int)(kh & 0xFFFFu);
        h = (int)(kh >> 16);
        const float2 r2 = S.r2[k];
        const float r = r2.x;
        // a list and the luminance limit need the exact codes of a passing pair
        const Intervals I = intervals32<FAST>(T, C, r2, S.sc4[h], A.half_w, A.clip);
        pc = certain_from(I, A.hi_min, A.lo_max, A.mask2, A.clip, DL);
        if (DL && pc > 0 && !dl_ok(A.ltab, A.max_dl, A.td[t].L, I.lo, I.lo + 3)) pc = 0;
        if (pc > 0) {
            if (acc.item.pb) {
                mark_pass(acc.item.pb, acc.item.k0, A.grid.H, k, h);
            } else {
                acc.cnt += inc;
                acc.rmax = fmaxf(acc.rmax, r);
                acc.pm |= 1u << pc;
            }
        }
    }
    __syncwarp();
    push_fp64(A, (int)lane < n && pc < 0, t, k, h, rq_t, rq_kh, rq_n, n_re, acc.item);
}


// One 32-slot step of a work item: every lane evaluates slot (k, h).  With
// CHECK, lanes past the item's last slot (active == false) contribute nothing.
// Returns true for a flagged FP32 slot (decided later by drain_flagged); the
// step itself never synchronises the warp.
template <int PREC, bool FAST, bool CHECK, bool CLIP, bool LIST, bool LINSEG, bool DL>
__device__ __forceinline__ bool slot_step(const SearchArgs& A, const Smem& S, const PairsT& P,
                                          const PairsC& PC, const TargetF64& D, int64_t t, int k,
                                          int h, bool active, Tally& acc) {
    const int H = A.grid.H;
    const int inc = A.grid.sym ? 2 : 1;
    if (CHECK && !active) { k = 0; h = 0; }
    const float2 r2 = S.r2[k];
    const float r = r2.x;
    if (PREC == CVS_PREC_FP32_RECHECK) {
        const float4 sc = S.sc4[h];
        const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y));  // (u, -u)
        const float2 w2 = __fmul2_rn(r2, f2(sc.z, sc.w));  // (w, -w)
        float2 lin[3];
        lin32<FAST>(P, PC, u2, w2, lin);
        if (!CLIP) {  // gamut reject: a warp whose pairs all leave the gamut is done
            const bool out = surely_out32(lin) || (CHECK && !active);
            if (__all_sync(0xFFFFFFFFu, out)) {
                acc.skip += (!CHECK || active) ? 1u : 0u;
                return false;
            }
        }
        int yp[3], ym[3];
        bool flag = encode32<LINSEG>(lin, A.half_w, yp, ym, nullptr);
        if (CHECK) flag = flag && active;
        int pattern = decide32<CLIP>(yp, ym, S.lut, A.mask2);
        if (flag || (CHECK && !active)) pattern = 0;
        if (DL && pattern) {
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
        if (pattern) {
            if (!LIST) {
                acc.cnt += inc;
                acc.rmax = fmaxf(acc.rmax, r);
                acc.pm |= 1u << pattern;  // bit p for pattern p; shifted down at the end
            } else {
                mark_pass(acc.item.pb, acc.item.k0, H, k, h);
            }
        }
        return flag;
    } else {
        int qp[3], qm[3];
        const int pattern = (!CHECK || active) ? decide64_slot(A, D, k, h, qp, qm) : 0;
        if (pattern) {
            if (LIST) {
                mark_pass(acc.item.pb, acc.item.k0, H, k, h);
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
static_assert(kSegIters <= kArcMaskWords, "a segment's start mask must fit its buffer");

// Iterations [it, end) of an item (within one segment starting at seg0), with
// lanes at slot (k, h); flagged slots set their bits in fb.
template <int PREC, bool FAST, bool CHECK, bool CLIP, bool LIST, bool LINSEG, bool DL>
__device__ __forceinline__ void run_range(const SearchArgs& A, const Smem& S, const PairsT& P,
                                          const PairsC& PC, const TargetF64& D, int64_t t, int& it,
                                          int end,
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
            const bool flag = slot_step<PREC, FAST, CHECK, CLIP, LIST, LINSEG, DL>(A, S, P, PC, D, t,
                                                                                 k, h, active, acc);
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
template <bool FAST, bool DL>
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
                drain_flagged<FAST, DL>(A, S, T, C, t, pq, 32, acc, rq_t, rq_kh, rq_n, n_re);
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

template <int PREC, bool FAST, bool CLIP, bool LIST, bool DL>
__device__ __forceinline__ void run_item(const SearchArgs& A, const Smem& S, int64_t t, int k0,
                                         int k1, const ChainF32& C, uint32_t* pq, uint32_t* fb,
                                         uint32_t* pb, uint32_t* rq_t, uint32_t* rq_kh, int& rq_n,
                                         unsigned long long& n_flag, unsigned long long& n_re,
                                         unsigned long long& n_skip,
                                         unsigned long long& n_prune) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    const int nslots = (k1 - k0) * H;
    TargetF32 T;
    TargetF64 D;
    if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
    if (PREC != CVS_PREC_FP32_RECHECK || DL) D = A.td[t];  // the limit needs the target's L*
    const PairsT P = make_pairs(T);
    const PairsC PC = make_pairs(C);
    Tally acc{0, -1.0f, 0u, 0u, 0u, ItemRef{pb, t, k0, k1}};
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
    if constexpr (PREC == CVS_PREC_FP32_RECHECK && FAST) {
        // iterations wholly below the first radius where a pair may pass are skipped
        const int k_pass = first_possible_radius(T, C, S.r2, k0, k1, A.hi_min);
        if (k_pass > k0) {
            it = k_pass == k1 ? nit : ((k_pass - k0) * H) >> 5;
            const int i = it * 32 + (int)lane;
            const int dk = i / H;
            k = k0 + dk;
            h = i - dk * H;
            if (lane == 0) acc.prune += k_pass == k1 ? (uint32_t)nslots : (uint32_t)(it * 32);
        }
    }
    for (int seg0 = it; seg0 < nit; seg0 += kSegIters) {
        const int seg1 = min(seg0 + kSegIters, nit);
        const int full_end = min(seg1, nfull);
        if constexpr (PREC == CVS_PREC_FP32_RECHECK && FAST) {
            run_range<PREC, FAST, false, CLIP, LIST, false, DL>(A, S, P, PC, D, t, it, min(full_end, it_pow),
                                                            seg0, nslots, q32, r32, k, h, acc, fb);
        }
        run_range<PREC, FAST, false, CLIP, LIST, true, DL>(A, S, P, PC, D, t, it, full_end, seg0, nslots,
                                                       q32, r32, k, h, acc, fb);
        if (it < seg1) {  // the item's last, partial iteration
            if (PREC == CVS_PREC_FP32_RECHECK && FAST && it < it_pow)
                run_range<PREC, FAST, true, CLIP, LIST, false, DL>(A, S, P, PC, D, t, it, seg1, seg0,
                                                               nslots, q32, r32, k, h, acc, fb);
            else
                run_range<PREC, FAST, true, CLIP, LIST, true, DL>(A, S, P, PC, D, t, it, seg1, seg0,
                                                              nslots, q32, r32, k, h, acc, fb);
        }
        if (PREC == CVS_PREC_FP32_RECHECK) {
            __syncwarp();
            collect_flagged<FAST, DL>(A, S, T, C, t, k0, seg0, (seg1 - seg0 + 31) >> 5, fb, pq, pq_n,
                                  acc, rq_t, rq_kh, rq_n, n_flag, n_re);
        }
    }
    if (PREC == CVS_PREC_FP32_RECHECK && pq_n > 0)
        drain_flagged<FAST, DL>(A, S, T, C, t, pq, pq_n, acc, rq_t, rq_kh, rq_n, n_re);
    n_skip += acc.skip;
    n_prune += acc.prune;
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

// List mode: words of a warp's passing-slot bitmap (an item has at most
// kListMaxSlots slots), and of the bitmap plus its nwords + 1 prefix counts in
// the emit kernel.
constexpr int kListWords = kListMaxSlots / 32;
constexpr int kListWarpWords = 2 * kListWords + 2 + 2 * kListMaxRadii;

// Queue the flagged slots of one segment of a list region (words [0, nwords)
// of fb; bit i of word w of lane l = position seg + 32 (32 w + i) + l) into
// pq, deciding each full batch of 32 with drain_flagged.
template <bool FAST, bool DL>
__device__ __forceinline__ void collect_list(const SearchArgs& A, const Smem& S, const ChainF32& C,
                                             int64_t t, int kg, const uint32_t* al, int jbeg,
                                             int jend, int seg, int nwords, uint32_t* fb,
                                             uint32_t* pq, int& pq_n, Tally& acc, uint32_t* rq_t,
                                             uint32_t* rq_kh, int& rq_n,
                                             unsigned long long& n_flag,
                                             unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const uint32_t* pos = al + kArcEntries;
    for (int w = 0; w < nwords; ++w) {
        uint32_t bits = fb[w * 32 + lane];
        fb[w * 32 + lane] = 0u;
        while (true) {
            const bool has = bits != 0u;
            const unsigned ball = __ballot_sync(0xFFFFFFFFu, has);
            if (!ball) break;
            if (has) {
                const int i = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int p = seg + 32 * (32 * w + i) + (int)lane;
                int lo = jbeg, hi = jend - 1;  // the last entry starting at or before p
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if ((int)pos[mid] <= p) lo = mid; else hi = mid - 1;
                }
                const uint32_t e = al[lo];
                const uint32_t k = (uint32_t)kg + (e & 127u);
                const uint32_t h = (uint32_t)(p + (int)(e >> 8) - kArcBias);
                pq[pq_n + __popc(ball & ((1u << lane) - 1u))] = k | (h << 16);
                ++n_flag;
            }
            pq_n += __popc(ball);
            __syncwarp();
            if (pq_n >= 32) {
                const TargetF32 T = A.tf[t];
                drain_flagged<FAST, DL>(A, S, T, C, t, pq, 32, acc, rq_t, rq_kh, rq_n, n_re);
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

// Positions [pbeg, pend) of a list region (entries jbeg .. jend - 1, entry
// jbeg starting at pbeg), 32 per step; the last, partial step is peeled.
// Flagged slots set their bits in fb and are collected after each segment of
// kSegIters steps.  The encode keeps its sRGB linear-segment select for every
// radius: one loop for the whole region.  (Two loops, split at the first
// radius that may reach the segment so that the radii below it skip the
// select, ran 2.3% slower: the kernel is bound by instruction issue and fetch,
// and the second loop doubled the hot code.)
template <bool FAST, bool LIST, bool DL>
__device__ __forceinline__ void run_list(const SearchArgs& A, const Smem& S, const PairsT& P,
                                         const PairsC& PC, const TargetF64& D, const ChainF32& C,
                                         int64_t t, int kg, uint32_t* al, int jbeg, int jend,
                                         int pbeg, int pend, Tally& acc, uint32_t* fb,
                                         uint32_t* pq, int& pq_n, uint32_t* rq_t, uint32_t* rq_kh,
                                         int& rq_n, unsigned long long& n_flag,
                                         unsigned long long& n_re) {
    constexpr int PREC = CVS_PREC_FP32_RECHECK;
    const unsigned lane = lane_id();
    const int pfull = pbeg + ((pend - pbeg) & ~31);  // start of the partial step
    int j0 = jbeg - 1;
    const uint32_t* msk = al + 2 * kArcEntries;
    for (int seg = pbeg; seg < pend; seg += 32 * kSegIters) {
        const int seg_end = min(pend, seg + 32 * kSegIters);
        list_mask(al, jend, seg, (seg_end - seg + 31) >> 5, j0);
        int b = seg;
        while (b < seg_end) {
            const int q = (b - seg) >> 5;  // step index within the segment
            const int w = q >> 5;
            const int wend = min(seg_end, seg + 1024 * (w + 1));
            uint32_t bits = 0, bit = 1u << (q & 31);
            for (; b < min(wend, pfull); b += 32) {
                const int p = b + (int)lane;
                const uint32_t e = list_step(al, msk[(b - seg) >> 5], j0);
                const int k = kg + (int)(e & 127u), h = p + (int)(e >> 8) - kArcBias;
                if (slot_step<PREC, FAST, false, false, LIST, true, DL>(A, S, P, PC, D, t, k, h,
                                                                        true, acc))
                    bits |= bit;
                bit <<= 1;
            }
            if (b < wend) {  // the partial step
                const int p = b + (int)lane;
                const bool active = p < pend;
                const uint32_t e = list_step(al, msk[(b - seg) >> 5], j0);
                const int k = kg + (int)(e & 127u), h = p + (int)(e >> 8) - kArcBias;
                if (slot_step<PREC, FAST, true, false, LIST, true, DL>(A, S, P, PC, D, t, k, h,
                                                                       active, acc))
                    bits |= bit;
                b = wend;
            }
            fb[w * 32 + lane] |= bits;
        }
        __syncwarp();
        const int nsteps = (seg_end - seg + 31) >> 5;
        collect_list<FAST, DL>(A, S, C, t, kg, al, jbeg, jend, seg, (nsteps + 31) >> 5, fb, pq,
                               pq_n, acc, rq_t, rq_kh, rq_n, n_flag, n_re);
    }
}

// A work item of the FP32 path (gamut reject) on a grid with angle ranges;
// see above.
template <bool LIST, bool DL>
__device__ __forceinline__ void run_item_arcs(const SearchArgs& A, const Smem& S, int64_t t,
                                              int k0, int k1, const ChainF32& C, uint32_t* pq,
                                              uint32_t* fb, uint32_t* al, uint32_t* pb, uint32_t* rq_t,
                                              uint32_t* rq_kh, int& rq_n,
                                              unsigned long long& n_flag,
                                              unsigned long long& n_re,
                                              unsigned long long& n_skip,
                                              unsigned long long& n_prune) {
    const unsigned lane = lane_id();
    const int H = A.grid.H, K = A.grid.K;
    TargetF64 D;
    if (DL) D = A.td[t];
    const PairsT P = make_pairs(A.tf[t]);
    const PairsC PC = make_pairs(C);
    Tally acc{0, -1.0f, 0u, 0u, 0u, ItemRef{pb, t, k0, k1}};
    int pq_n = 0;
    uint32_t* pos = al + kArcEntries;
    const uint2* ranges = A.arc_ranges + t * K;
    for (int kb = k0; kb < k1; kb += kArcRadii) {
        const int kb1 = min(k1, kb + kArcRadii);
        // the list: the fast-path radii's ranges (entries [0, js), positions
        // [0, ps)), then the slow-path radii's (to nf and pf)
        int nf = 0, pf = 0, js = 0, ps = 0;
        for (int region = 0; region < 2; ++region) {
            for (int kg = kb; kg < kb1; kg += 32) {
                const int k = kg + (int)lane;
                const uint2 o = k < kb1 ? ranges[k] : make_uint2(0u, 0u);
                const bool take = k < kb1 && ((o.x & kSlowRadius) != 0u) == (region == 1);
                const uint32_t w0 = take ? (o.x & ~kSlowRadius) : 0u, w1 = take ? o.y : 0u;
                const int l0 = (int)(w0 >> 16), l1 = (int)(w1 >> 16);
                const int n = (l0 > 0 ? 1 : 0) + (l1 > 0 ? 1 : 0);
                const int tot = l0 + l1;
                if (take) acc.prune += (uint32_t)(H - tot);
                int nr, pr;
                const int eoff = nf + warp_exclusive_sum(n, nr);
                const int poff = pf + warp_exclusive_sum(tot, pr);
                const uint32_t koff = (uint32_t)(k - kb);
                int e = eoff, q = poff;
                if (l0 > 0) {
                    al[e] = koff | ((uint32_t)((int)(w0 & 0xFFFFu) - q + kArcBias) << 8);
                    pos[e] = (uint32_t)q;
                    ++e;
                    q += l0;
                }
                if (l1 > 0) {
                    al[e] = koff | ((uint32_t)((int)(w1 & 0xFFFFu) - q + kArcBias) << 8);
                    pos[e] = (uint32_t)q;
                }
                nf += nr;
                pf += pr;
            }
            if (region == 0) {
                js = nf;
                ps = pf;
            }
        }
        if (lane == 0) pos[nf] = (uint32_t)pf;  // (pos[js] = ps: the first slow entry or this)
        __syncwarp();
        run_list<true, LIST, DL>(A, S, P, PC, D, C, t, kb, al, 0, js, 0, ps, acc, fb, pq, pq_n,
                                 rq_t, rq_kh, rq_n, n_flag, n_re);
        if (nf > js) {  // the slow path decides its own flagged slots
            if (pq_n > 0) {
                const TargetF32 T = A.tf[t];
                drain_flagged<true, DL>(A, S, T, C, t, pq, pq_n, acc, rq_t, rq_kh, rq_n, n_re);
                pq_n = 0;
            }
            run_list<false, LIST, DL>(A, S, P, PC, D, C, t, kb, al, js, nf, ps, pf, acc, fb, pq,
                                      pq_n, rq_t, rq_kh, rq_n, n_flag, n_re);
            if (pq_n > 0) {
                const TargetF32 T = A.tf[t];
                drain_flagged<false, DL>(A, S, T, C, t, pq, pq_n, acc, rq_t, rq_kh, rq_n, n_re);
                pq_n = 0;
            }
        }
        __syncwarp();  // the list is rebuilt for the next block of radii
    }
    if (pq_n > 0) {
        const TargetF32 T = A.tf[t];
        drain_flagged<true, DL>(A, S, T, C, t, pq, pq_n, acc, rq_t, rq_kh, rq_n, n_re);
    }
    n_skip += acc.skip;
    n_prune += acc.prune;
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

// The slot ranges of a chunk of targets (see run_item_arcs): one warp per
// target, lanes over its radii.
#ifndef CVS_ARC_PASS_MIN_BLOCKS
#define CVS_ARC_PASS_MIN_BLOCKS 3
#endif
template <bool CLIP>
__global__ void __launch_bounds__(256, CVS_ARC_PASS_MIN_BLOCKS)
    k_arc_ranges(const SearchArgs A, int64_t nt, uint2* __restrict__ out,
                             unsigned long long* __restrict__ probe, int64_t stride) {
    ChainF32 C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C.Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        C.Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    uint32_t chm = 0;
#pragma unroll
    for (int p = 1; p < 8; ++p) chm |= ((A.mask2 >> p) & 1u) ? (uint32_t)p : 0u;
    const int K = A.grid.K, H = A.grid.H;
    const unsigned lane = lane_id();
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long covered = 0, plain = 0;  // probe: slots listed / walked without ranges
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt;
         t += nwarps) {
        const TargetF32 T = A.tf[t * stride];
        for (int k = (int)lane; k < K; k += 32) {
            const float r = __ldg(A.grid.r32 + k);
            const bool slow = !((T.flags & 1u) || fast_radius(T, r));
            uint2 o;
            uint32_t rr[kMaxArcRanges];
            int tot = 0;
            const int n = radius_ranges_body<CLIP>(T, C, r, A.hi_min, chm, A.grid.th0,
                                                   A.grid.inv_step, H, rr, tot);
            o.x = n > 0 ? rr[0] : 0u;
            o.y = 0u;
            if (n == 2) o.y = rr[1];
            if (n > 2) {  // cover the second to the last range with one
                const uint32_t s1 = rr[1] & 0xFFFFu, last = rr[n - 1];
                const uint32_t e = (last & 0xFFFFu) + (last >> 16);
                o.y = s1 | ((e - s1) << 16);
            }
            if (slow) o.x |= kSlowRadius;
            if (probe) {  // the plain walk searches a slow-path radius whole
                covered += tot;
                plain += (!slow && certain_fail_radius(T, C, r, A.hi_min)) ? 0 : H;
            }
            out[t * K + k] = o;
        }
    }
    if (probe) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            covered += __shfl_xor_sync(0xFFFFFFFFu, covered, off);
            plain += __shfl_xor_sync(0xFFFFFFFFu, plain, off);
        }
        if (lane == 0 && plain) {
            atomicAdd(probe, covered);
            atomicAdd(probe + 1, plain);
        }
    }
}

// ------------------------------------------------------------ pair-list output
// A pair list takes three kernels per batch of colours.  The search (list
// mode) leaves, per work item g, the bitmap of its passing slots in item_bits
// (item_words words from g * item_words) and their number in item_count[g], and
// goes on with its next item.  k_scan_tiles / k_scan_top turn the counts into
// the position of every item's first record.  k_emit_pairs then writes the
// records of every item straight to their place (see emit_records).  Records of
// an item follow those of every earlier item, which is (target, k, m) order.

// The end of a list-mode work item: its bitmap and count to global memory (one
// coalesced row), and the shared bitmap cleared for the next item.
__device__ __forceinline__ void store_item(const SearchArgs& A, long long g, int nwords,
                                           uint32_t* pb) {
    const unsigned lane = lane_id();
    uint32_t* dst = A.item_bits + g * (long long)A.item_words;
    int cnt = 0;
    for (int w = (int)lane; w < nwords; w += 32) {
        const uint32_t v = pb[w];
        dst[w] = v;
        cnt += __popc(v);
        pb[w] = 0u;
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt);
    if (lane == 0) A.item_count[g] = (uint32_t)cnt;
    __syncwarp();
}

// Launch bounds of the search kernel: blocks of up to CVS_SEARCH_MAX_THREADS
// threads, at least CVS_SEARCH_MIN_BLOCKS of them resident per SM.
#ifndef CVS_SEARCH_MAX_THREADS
#define CVS_SEARCH_MAX_THREADS kSearchBlock
#endif
#ifndef CVS_SEARCH_MIN_BLOCKS
#define CVS_SEARCH_MIN_BLOCKS 6
#endif
#ifndef CVS_ARCS_MIN_BLOCKS
#define CVS_ARCS_MIN_BLOCKS 7  // 6 measured 2.9% slower, 8 (with halved segments to fit) 7%
#endif

// ARCS: the angle-range walk (FP32, gamut reject, a grid with angle ranges),
// a separate instantiation so that the plain walk's code and registers stay
// as they are without it.  (ARCS = false compiles no range walk at all.)
template <int PREC, bool CLIP, bool LIST, bool DL, bool ARCS>
__global__ void __launch_bounds__(CVS_SEARCH_MAX_THREADS,
                                  ARCS ? CVS_ARCS_MIN_BLOCKS : CVS_SEARCH_MIN_BLOCKS)
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
    uint32_t* al = S.rq_kh + 2 * nwarps * kRqCap + nwarps * (kFlagWords * 32) + warp * kArcWords;
    // list mode: per warp the item's passing-slot bitmap
    uint32_t* pb = nullptr;
    if (LIST) {
        pb = S.rq_kh + 2 * nwarps * kRqCap + nwarps * (kFlagWords * 32) +
             (A.grid.arcs ? nwarps * kArcWords : 0) + warp * kListWords;
        for (int w = lane_id(); w < kListWords; w += 32) pb[w] = 0u;
    }
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
    unsigned long long n_flag = 0, n_re = 0, n_skip = 0, n_prune = 0;
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
        // (a run-time test: the plain walk stays compiled into the range
        // kernel, which measured faster than without it)
        if (ARCS && PREC == CVS_PREC_FP32_RECHECK && !CLIP && A.grid.arcs) {
            run_item_arcs<LIST, DL>(A, S, t, k0, k1, C, pq, fb, al, pb, rq_t, rq_kh, rq_n, n_flag,
                                    n_re, n_skip, n_prune);
        } else if (PREC == CVS_PREC_FP32_RECHECK) {
            const uint32_t fl = A.tf[t].flags;
            if (fl & 1u)
                run_item<PREC, true, CLIP, LIST, DL>(A, S, t, k0, k1, C, pq, fb, pb, rq_t, rq_kh, rq_n,
                                                     n_flag, n_re, n_skip, n_prune);
            else
                run_item<PREC, false, CLIP, LIST, DL>(A, S, t, k0, k1, C, pq, fb, pb, rq_t, rq_kh,
                                                      rq_n, n_flag, n_re, n_skip, n_prune);
        } else {
            run_item<PREC, true, CLIP, LIST, DL>(A, S, t, k0, k1, C, pq, fb, pb, rq_t, rq_kh, rq_n,
                                                 n_flag, n_re, n_skip, n_prune);
        }
        // list mode: the item's bitmap and count (slots still queued for FP64
        // reach them in global memory when the queue is flushed)
        if (LIST) store_item(A, A.item0 + (long long)item, ((k1 - k0) * H + 31) >> 5, pb);
    }
    if (PREC == CVS_PREC_FP32_RECHECK && rq_n > 0)
        flush_queue(A, rq_t, rq_kh, rq_n, &n_re, nullptr, -1, 0, 0);
    // statistics
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n_flag += __shfl_xor_sync(0xFFFFFFFFu, n_flag, off);
        n_re += __shfl_xor_sync(0xFFFFFFFFu, n_re, off);
        n_skip += __shfl_xor_sync(0xFFFFFFFFu, n_skip, off);
        n_prune += __shfl_xor_sync(0xFFFFFFFFu, n_prune, off);
    }
    if (lane == 0) {
        if (n_flag) atomicAdd(A.stats + 0, n_flag);
        if (n_re) atomicAdd(A.stats + 1, n_re);
        if (n_skip) atomicAdd(A.stats + 3, n_skip);
        if (n_prune) atomicAdd(A.stats + 4, n_prune);
    }
}

// ------------------------------------------------------------ pair-list records
// FP32 codes of slot (k, h) of a target for its record; returns true when
// some code lies within the window W of a rounding boundary (the record then
// takes FP64 codes, see flush_records).
__device__ __forceinline__ bool record_codes32(const EmitArgs& A, const float2* r2s,
                                               const float4* sc4s, const ChainF32& C,
                                               const TargetF32& T, int k, int h, int qp[3],
                                               int qm[3]) {
    const float2 r2 = r2s[k];
    const float4 sc = sc4s[h];
    const PairsT P = make_pairs(T);
    const PairsC PC = make_pairs(C);
    const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y)), w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
    int yp[3], ym[3];
    const bool flag = ((T.flags & 1u) || fast_radius(T, r2.x))
                          ? codes32<true>(P, PC, u2, w2, A.half_w, yp, ym)
                          : codes32<false>(P, PC, u2, w2, A.half_w, yp, ym);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        qp[c] = yp[c] - kMagicBits;
        qm[c] = ym[c] - kMagicBits;
    }
    return flag;
}

// Store the record of slot (k, h) at pos (if below the capacity) and, on a
// folded grid, its +180 degree partner at pos + ck; codes clamped in clip mode.
__device__ __forceinline__ void store_records(const EmitArgs& A, uint32_t target, int k, int h,
                                              int qp_in[3], int qm_in[3], uint32_t fp64,
                                              unsigned long long pos, unsigned ck) {
    int qp[3], qm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        qp[c] = A.clip ? min(max(qp_in[c], 0), 255) : qp_in[c];
        qm[c] = A.clip ? min(max(qm_in[c], 0), 255) : qm_in[c];
    }
    Decide dc;
    dc.hi_min = A.hi_min;
    dc.lo_max = A.lo_max;
    dc.mask2 = A.mask2;
    dc.clip = A.clip;
    const int pattern = decide_codes(qp, qm, dc);
    const uint32_t tail = (uint32_t)pattern << 16 | fp64 << 24;
    uint4* out = reinterpret_cast<uint4*>(A.out);
    if (pos < (unsigned long long)A.out_cap)
        out[pos] = make_uint4((uint32_t)k | (uint32_t)h << 16,
                              (uint32_t)qp[0] | (uint32_t)qp[1] << 8 | (uint32_t)qp[2] << 16 |
                                  (uint32_t)qm[0] << 24,
                              (uint32_t)qm[1] | (uint32_t)qm[2] << 8 | tail, target);
    if (A.grid.sym && pos + ck < (unsigned long long)A.out_cap)
        out[pos + ck] = make_uint4((uint32_t)k | (uint32_t)(h + A.grid.H) << 16,
                                   (uint32_t)qm[0] | (uint32_t)qm[1] << 8 |
                                       (uint32_t)qm[2] << 16 | (uint32_t)qp[0] << 24,
                                   (uint32_t)qp[1] | (uint32_t)qp[2] << 8 | tail, target);
}

// Records whose codes need FP64, queued per warp: the position, the partner's
// offset and the slot.  They are computed 32 at a time, one per lane, so the
// FP64 pipe runs full warps.
struct RecQueue {
    unsigned long long* pos;
    uint32_t* ck;
    uint32_t* kh;
    uint32_t* t;  // the target (index within the batch)
    int n;        // queued entries (warp-uniform); the queue runs across items
};
constexpr int kRecQueue = 64;

__device__ __noinline__ void flush_records(const EmitArgs& A, const RecQueue& Q, int n) {
    const unsigned lane = lane_id();
    if ((int)lane < n) {
        const uint32_t kh = Q.kh[lane], t = Q.t[lane];
        const int k = (int)(kh & 0xFFFFu), h = (int)(kh >> 16);
        const TargetF64 D = A.td[t];
        int qp[3], qm[3];
        pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + k), __ldg(A.grid.s64 + h),
                     __ldg(A.grid.c64 + h), A.qkey, qp, qm);
        store_records(A, A.target_id + t, k, h, qp, qm, 1u, Q.pos[lane], Q.ck[lane]);
    }
    __syncwarp();
}

// Passing slots of an item's bitmap before slot s (pre: exclusive prefix of
// the words' counts, nwords + 1 entries).
__device__ __forceinline__ int passing_before(const uint32_t* pb, const uint32_t* pre, int s) {
    const int w = s >> 5, b = s & 31;
    return (int)pre[w] + (b ? __popc(pb[w] & ((1u << b) - 1u)) : 0);
}

// Positions of the items' records: k_scan_tiles gives, per tile of kScanTile
// items, each item's records before it within the tile and the tile's total;
// k_scan_top the records before each tile (after the carry: the records of the
// earlier batches, offs[0]).  An item has (passing slots) << sym records.
constexpr int kScanTile = 4096;
__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* __restrict__ count, int sym,
                                                     int64_t n, int64_t* __restrict__ within,
                                                     int64_t* __restrict__ tile_sum) {
    __shared__ long long warp_sum[32];
    const int64_t i0 = (int64_t)blockIdx.x * kScanTile + 4 * (int64_t)threadIdx.x;
    long long v[4], run = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = i0 + j < n ? (long long)count[i0 + j] << sym : 0;
        run += v[j];
    }
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    long long x = run;  // inclusive scan of the threads' sums within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if ((int)lane >= off) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = warp_sum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long y = __shfl_up_sync(0xFFFFFFFFu, w, off);
            if ((int)lane >= off) w += y;
        }
        warp_sum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    long long ex = x - run + (warp > 0 ? warp_sum[warp - 1] : 0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) within[i0 + j] = ex;
        ex += v[j];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = warp_sum[31];
}

__global__ void __launch_bounds__(1024) k_scan_top(int64_t* __restrict__ tile, int ntiles,
                                                   const int64_t* __restrict__ carry) {
    __shared__ long long warp_sum[32];
    __shared__ long long base;
    if (threadIdx.x == 0) base = carry[0];
    __syncthreads();
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    for (int t0 = 0; t0 < ntiles; t0 += 1024) {
        const int t = t0 + (int)threadIdx.x;
        const long long v = t < ntiles ? tile[t] : 0;
        long long x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if ((int)lane >= off) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long y = __shfl_up_sync(0xFFFFFFFFu, w, off);
                if ((int)lane >= off) w += y;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        const long long ex = base + x - v + (warp > 0 ? warp_sum[warp - 1] : 0);
        if (t < ntiles) tile[t] = ex;  // in place: records before tile t
        __syncthreads();
        if (threadIdx.x == 0) base += warp_sum[31];
        __syncthreads();
    }
}

// The records of one item (target t, radii [k0, k1), its bitmap pb with word
// prefixes pre, first record at base): per radius k its passing slots in
// ascending h with m = h, then, on a folded grid, the same slots again with
// m = h + H and the colours swapped.  Lane j of a round takes the j-th next
// passing slot, so consecutive lanes store consecutive 16-byte records;
// records whose FP32 codes are flagged wait in the warp's queue for FP64.
// Records at or beyond A.out_cap are not written.
template <int PREC>
__device__ __forceinline__ void emit_records(const EmitArgs& A, const float2* r2s,
                                             const float4* sc4s, const ChainF32& C, int64_t t,
                                             int k0, int nwords, int P, long long base,
                                             const uint32_t* pb, const uint32_t* pre,
                                             const uint32_t* rad, RecQueue& Q) {
    const unsigned lane = lane_id();
    const int H = A.grid.H, sym = A.grid.sym;
    TargetF32 T{};
    if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
    const uint32_t target = A.target_id + (uint32_t)t;
    for (int r0 = 0; r0 < P; r0 += 32) {
        const int R = r0 + (int)lane;
        bool need64 = false;
        int k = 0, h = 0;
        unsigned long long pos = 0;
        unsigned ck = 0;
        if (R < P) {
            int lo = 0, hi = nwords - 1;  // the word holding the R-th passing slot
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int)pre[mid] <= R) lo = mid; else hi = mid - 1;
            }
            const int s = lo * 32 + (int)__fns(pb[lo], 0, R - (int)pre[lo] + 1);
            const int dk = s / H;
            h = s - dk * H;
            k = k0 + dk;
            const int before = (int)rad[2 * dk];  // passing slots of earlier radii, this one's
            ck = rad[2 * dk + 1];
            pos = (unsigned long long)base + ((unsigned long long)before << sym) +
                  (unsigned)(R - before);
            if (PREC == CVS_PREC_FP32_RECHECK) {
                int qp[3], qm[3];
                need64 = record_codes32(A, r2s, sc4s, C, T, k, h, qp, qm);
                if (!need64) store_records(A, target, k, h, qp, qm, 0u, pos, ck);
            } else {
                need64 = true;
            }
        }
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, need64);
        if (need64) {
            const int slot = Q.n + __popc(ball & ((1u << lane) - 1u));
            Q.pos[slot] = pos;
            Q.ck[slot] = ck;
            Q.kh[slot] = (uint32_t)k | (uint32_t)h << 16;
            Q.t[slot] = (uint32_t)t;
        }
        Q.n += __popc(ball);
        __syncwarp();
        if (Q.n >= 32) {
            flush_records(A, Q, 32);
            const int rest = Q.n - 32;  // below kRecQueue - 32
            unsigned long long mp = 0;
            uint32_t mc = 0, mk = 0, mt = 0;
            if ((int)lane < rest) {
                mp = Q.pos[32 + lane];
                mc = Q.ck[32 + lane];
                mk = Q.kh[32 + lane];
                mt = Q.t[32 + lane];
            }
            __syncwarp();
            if ((int)lane < rest) {
                Q.pos[lane] = mp;
                Q.ck[lane] = mc;
                Q.kh[lane] = mk;
                Q.t[lane] = mt;
            }
            __syncwarp();
            Q.n = rest;
        }
    }
}

// One warp per work item (grid-stride): stage the item's bitmap in shared
// memory, scan its words, set the per-target offsets, write the records.
template <int PREC>
__global__ void __launch_bounds__(kSearchBlock) k_emit_pairs(const EmitArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H;
    float2* r2s = reinterpret_cast<float2*>(smem);
    float4* sc4s = reinterpret_cast<float4*>(smem + ((K * 8 + 15) & ~15));
    unsigned char* per_warp = smem + ((K * 8 + 15) & ~15) + H * 16;
    const int warp = threadIdx.x >> 5;
    RecQueue Q;  // per warp: positions (8 B), partner offsets, slots, targets (4 B each)
    Q.pos = reinterpret_cast<unsigned long long*>(per_warp) + warp * kRecQueue;
    Q.ck = reinterpret_cast<uint32_t*>(per_warp + (kSearchBlock / 32) * kRecQueue * 8) +
           warp * 3 * kRecQueue;
    Q.kh = Q.ck + kRecQueue;
    Q.t = Q.kh + kRecQueue;
    Q.n = 0;
    uint32_t* pb = reinterpret_cast<uint32_t*>(per_warp + (kSearchBlock / 32) * kRecQueue * 20) +
                   warp * kListWarpWords;
    uint32_t* pre = pb + kListWords;
    uint32_t* rad = pre + kListWords + 2;  // per radius of the item: (passing before, count)
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
    const unsigned lane = lane_id();
    const int n_kc = (K + A.kchunk - 1) / A.kchunk;
    const long long n_items = A.n_targets * (long long)n_kc;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_items;
         g += nwarps) {
        const int64_t t = g / n_kc;
        const int kc = (int)(g - t * n_kc);
        const int k0 = kc * A.kchunk, k1 = min(k0 + A.kchunk, K);
        const int nwords = ((k1 - k0) * H + 31) >> 5;
        const uint32_t* src = A.item_bits + g * (long long)A.item_words;
        int run = 0;
        for (int w0 = 0; w0 < nwords; w0 += 32) {
            const int w = w0 + (int)lane;
            const uint32_t v = w < nwords ? src[w] : 0u;
            if (w < nwords) pb[w] = v;
            int tot;
            const int ex = warp_exclusive_sum(__popc(v), tot);
            if (w < nwords) pre[w] = (uint32_t)(run + ex);
            run += tot;
        }
        if (lane == 0) pre[nwords] = (uint32_t)run;
        __syncwarp();
        for (int dk = (int)lane; dk < k1 - k0; dk += 32) {  // per radius: passing before, count
            const int b0 = passing_before(pb, pre, dk * H);
            rad[2 * dk] = (uint32_t)b0;
            rad[2 * dk + 1] = (uint32_t)(passing_before(pb, pre, dk * H + H) - b0);
        }
        __syncwarp();
        const long long base = A.tile_base[g / kScanTile] + A.item_base[g];
        if (lane == 0) {
            if (kc == 0) A.offs[t] = base;
            if (kc == n_kc - 1) A.offs[t + 1] = base + ((long long)run << A.grid.sym);
        }
        emit_records<PREC>(A, r2s, sc4s, C, t, k0, nwords, run, base, pb, pre, rad, Q);
        __syncwarp();
    }
    if (Q.n > 0) flush_records(A, Q, Q.n);
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

// ------------------------------------------------------------ L* of all colours
__global__ void k_l_table(double* __restrict__ ltab) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ((int64_t)1 << 24)) return;
    double L, a, b;
    target_lab64((uint32_t)(i >> 16), (uint32_t)(i >> 8) & 255u, (uint32_t)i & 255u, L, a, b);
    ltab[i] = L;
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
// Every (target, k, m) plus colour in FP32 (each chain the search may take for
// it: the cubic-branch chain where the target or the radius stays on the cubic
// branch of f^-1, the branchy chain for targets that may leave it) against the
// FP64 chain.  Per value, exactly: the FP32 code round(v32) against the FP64
// code (threshold count), and whether the search would flag it (v32 within W of
// a rounding boundary, |v32 - round(v32)| >= half_w).  Counts: out[0] FP32
// codes in [-1, 256] that differ from FP64, out[1] those among them the search
// would take unflagged (must be 0 for exact results), out[2] values examined.
// Maxima (float bits): |lin32 - lin64|; |v32 - v64| among values with v64
// within 0.05 of a boundary (v64 by the FP64 power, evaluated only where v32
// lies within 0.08 of a boundary; with |lin32 - lin64| small that covers every
// such value); the a*/b* error of the colour the FP32 chain stands for.
// One warp per target (grid-stride), lanes over the K x N values.
__global__ void k_precision_probe(const TargetF32* __restrict__ tf, const TargetF64* __restrict__ td,
                                  int64_t n, const GridDev g, const long long* __restrict__ qkey,
                                  float half_w, unsigned int* max_v_err_bits,
                                  unsigned int* max_lin_err_bits, unsigned int* max_lab_err_bits,
                                  unsigned long long* counts) {
    float Ax[3], Bz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    const unsigned lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int KN = g.K * g.N;
    float vmax = 0.0f, lmax = 0.0f, amax = 0.0f;
    unsigned long long wrong = 0, unflagged_wrong = 0, values = 0;
    for (int64_t t = warp; t < n; t += nwarps) {
        const TargetF32 T = tf[t];
        const TargetF64 D = td[t];
        const PairsT P = make_pairs(T);
        const double fy = __ddiv_rn(__dadd_rn(D.L, 16.0), 116.0);
        for (int i = (int)lane; i < KN; i += 32) {
            const int k = i / g.N, m = i - k * g.N;
            const float r = g.r32[k];
            const float2 sc = g.sc32[m];
            const double da = __dmul_rn(g.r64[k], g.s64[m]), db = __dmul_rn(g.r64[k], g.c64[m]);
            double lin[3];
            color_lin64(D.L, __dadd_rn(D.a, da), __dadd_rn(D.b, db), lin);
            int q64[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) q64[c] = quantize64(lin[c], qkey);
            const float u = r * sc.x, w = r * sc.y;
            {  // a*, b* of the colour the FP32 chain stands for: f-values fx0 + u, fz0 + w
                const double fx_exact = fy + (D.a + da) * 0.002, fz_exact = fy - (D.b + db) * 0.005;
                const double ea = 500.0 * fabs(((double)T.fx0 + (double)u) - fx_exact);
                const double eb = 200.0 * fabs(((double)T.fz0 + (double)w) - fz_exact);
                amax = fmaxf(amax, (float)fmax(ea, eb));
            }
            const bool fast_ok = (T.flags & 1u) || fast_radius(T, r);
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 0 && !fast_ok) continue;     // the cubic-branch chain
                if (pass == 1 && (T.flags & 1u)) continue;  // the branchy chain
                float2 dX2, dZ2;
                if (pass == 0) delta_xz<true>(P, f2(u, -u), f2(w, -w), dX2, dZ2);
                else delta_xz<false>(P, f2(u, -u), f2(w, -w), dX2, dZ2);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float l32 = __ffma2_rn(f2(Bz[c], Bz[c]), dZ2,
                                                 __ffma2_rn(f2(Ax[c], Ax[c]), dX2,
                                                            f2(T.lin0[c], T.lin0[c]))).x;
                    const float v32 = encode_v32(l32);
                    const float d = v32 - rintf(v32);
                    const int q32 = (int)fminf(fmaxf(rintf(v32), -1.0f), 256.0f);
                    lmax = fmaxf(lmax, (float)fabs((double)l32 - lin[c]));
                    if (q32 != q64[c]) {
                        ++wrong;
                        if (fabsf(d) < half_w) ++unflagged_wrong;
                    }
                    if (fabsf(d) > 0.42f && v32 > -2.0f && v32 < 258.0f) {
                        const double l64 = lin[c];
                        const double v64 = l64 <= 0.0031308 ? 3294.6 * l64
                                                            : 269.025 * pow(l64, 1.0 / 2.4) - 14.025;
                        const double frac = v64 - floor(v64);
                        if (fabs(frac - 0.5) < 0.05) vmax = fmaxf(vmax, (float)fabs((double)v32 - v64));
                    }
                    ++values;
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        vmax = fmaxf(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, off));
        lmax = fmaxf(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, off));
        amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, off));
        wrong += __shfl_xor_sync(0xFFFFFFFFu, wrong, off);
        unflagged_wrong += __shfl_xor_sync(0xFFFFFFFFu, unflagged_wrong, off);
        values += __shfl_xor_sync(0xFFFFFFFFu, values, off);
    }
    if (lane == 0) {
        atomicMax(max_v_err_bits, __float_as_uint(vmax));
        atomicMax(max_lin_err_bits, __float_as_uint(lmax));
        atomicMax(max_lab_err_bits, __float_as_uint(amax));
        if (wrong) atomicAdd(counts, wrong);
        if (unflagged_wrong) atomicAdd(counts + 1, unflagged_wrong);
        if (values) atomicAdd(counts + 2, values);
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

int search_smem_bytes(const GridDev& g, int block, int list) {
    // (r, r) pairs, angle quadruples, then per warp: FP64 queue (targets, slots)
    // and flagged queue, on grids with angle ranges the range list, and in list
    // mode the item's bitmap with its prefix counts
    return ((g.K * 8 + 15) & ~15) + g.H * 16 + 3 * 512 +
           (block / 32) * (kRqCap * 12 + kFlagWords * 32 * 4 + (g.arcs ? kArcWords * 4 : 0) +
                           (list ? kListWords * 4 : 0));
}

template <int PREC, bool CLIP, bool LIST, bool DL>
cudaError_t launch_search_t(const SearchArgs& a_in, cudaStream_t st) {
    SearchArgs a = a_in;
    // (in clip mode only the high arcs prune, too few slots to pay for the walk)
    const bool arcs = PREC == CVS_PREC_FP32_RECHECK && !CLIP && a.grid.arcs && a.arc_ranges &&
                      a.arc_cap >= a.grid.K;
    a.grid.arcs = arcs ? 1 : 0;
    const int smem = search_smem_bytes(a.grid, a.shape.block, LIST);
    constexpr bool kArcsKernel = PREC == CVS_PREC_FP32_RECHECK && !CLIP;
    const void* fn = arcs ? (const void*)k_search<PREC, CLIP, LIST, DL, kArcsKernel>
                          : (const void*)k_search<PREC, CLIP, LIST, DL, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = a.shape.blocks_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, a.shape.block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    if (!arcs) {
        k_search<PREC, CLIP, LIST, DL, false><<<a.num_sms * per_sm, a.shape.block, smem, st>>>(a);
        return cudaGetLastError();
    }
    // angle ranges: per chunk of targets, the ranges pass, then the search
    const int64_t chunk = a.arc_cap / a.grid.K;
    for (int64_t t0 = 0; t0 < a_in.n_targets; t0 += chunk) {
        const int64_t nt = a_in.n_targets - t0 < chunk ? a_in.n_targets - t0 : chunk;
        SearchArgs c = a;
        c.tf += t0;
        c.td += t0;
        c.acc += t0;
        c.n_targets = nt;
        c.target_id = a.target_id + (uint32_t)t0;
        if (LIST)  // items of this chunk follow those of the earlier chunks
            c.item0 = a.item0 + t0 * ((a.grid.K + a.shape.kchunk - 1) / a.shape.kchunk);
        if (t0 > 0) {
            e = cudaMemsetAsync(c.work_counter, 0, sizeof(unsigned long long), st);
            if (e != cudaSuccess) return e;
        }
        const int64_t want = (nt + 7) / 8, cap = (int64_t)a.num_sms * 16;  // 8 warps a block
        k_arc_ranges<false><<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(
            c, nt, c.arc_ranges, nullptr, 1);
        if (t0 == 0 && a.ev_ranges) {
            e = cudaEventRecordWithFlags((cudaEvent_t)a.ev_ranges, st, a.ev_flags);
            if (e != cudaSuccess) return e;
        }
        k_search<PREC, CLIP, LIST, DL, kArcsKernel><<<a.num_sms * per_sm, a.shape.block, smem, st>>>(
            c);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int PREC, bool DL>
cudaError_t launch_search_d(const SearchArgs& a, cudaStream_t st) {
    if (a.clip) return a.list_mode ? launch_search_t<PREC, true, true, DL>(a, st)
                                   : launch_search_t<PREC, true, false, DL>(a, st);
    return a.list_mode ? launch_search_t<PREC, false, true, DL>(a, st)
                       : launch_search_t<PREC, false, false, DL>(a, st);
}

template <int PREC>
cudaError_t launch_search_p(const SearchArgs& a, cudaStream_t st) {
    return a.ltab ? launch_search_d<PREC, true>(a, st) : launch_search_d<PREC, false>(a, st);
}

cudaError_t launch_arc_probe(const SearchArgs& a, int64_t nt, int64_t stride,
                             unsigned long long* counts, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess || nt <= 0) return e;
    const int64_t want = (nt + 7) / 8, cap = (int64_t)a.num_sms * 16;
    k_arc_ranges<false><<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(a, nt, a.arc_ranges,
                                                                            counts, stride);
    return cudaGetLastError();
}

cudaError_t launch_arc_pass(const SearchArgs& a, int64_t nt, uint2* out, cudaStream_t st) {
    if (nt <= 0) return cudaSuccess;
    const int64_t want = (nt + 7) / 8, cap = (int64_t)a.num_sms * 16;  // 8 warps a block
    k_arc_ranges<false><<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(a, nt, out, nullptr,
                                                                            1);
    return cudaGetLastError();
}

cudaError_t launch_search(const SearchArgs& a, cudaStream_t st) {
    return a.prec == CVS_PREC_FP64 ? launch_search_p<CVS_PREC_FP64>(a, st)
                                   : launch_search_p<CVS_PREC_FP32_RECHECK>(a, st);
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

cudaError_t launch_pair_scan(const uint32_t* count, int sym, int64_t n_items, int64_t* within,
                             int64_t* tile, const int64_t* carry, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const int64_t ntiles = (n_items + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<(unsigned)ntiles, 1024, 0, st>>>(count, sym, n_items, within, tile);
    k_scan_top<<<1, 1024, 0, st>>>(tile, (int)ntiles, carry);
    return cudaGetLastError();
}

int emit_smem_bytes(const GridDev& g) {
    // tables, then per warp the record queue (16 B an entry) and the bitmap
    // with its prefix counts
    return ((g.K * 8 + 15) & ~15) + g.H * 16 +
           (kSearchBlock / 32) * (kRecQueue * 20 + kListWarpWords * 4);
}

cudaError_t launch_emit_pairs(const EmitArgs& a, int num_sms, cudaStream_t st) {
    const int64_t n_items = a.n_targets * ((a.grid.K + a.kchunk - 1) / a.kchunk);
    if (n_items <= 0) return cudaSuccess;
    const int smem = emit_smem_bytes(a.grid);
    const void* fn = a.prec == CVS_PREC_FP64 ? (const void*)k_emit_pairs<CVS_PREC_FP64>
                                             : (const void*)k_emit_pairs<CVS_PREC_FP32_RECHECK>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t want = (n_items + 3) / 4, cap = (int64_t)num_sms * 16;  // 4 warps a block
    const unsigned blocks = (unsigned)(want < cap ? want : cap);
    if (a.prec == CVS_PREC_FP64)
        k_emit_pairs<CVS_PREC_FP64><<<blocks, kSearchBlock, smem, st>>>(a);
    else
        k_emit_pairs<CVS_PREC_FP32_RECHECK><<<blocks, kSearchBlock, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_l_table(double* ltab, cudaStream_t st) {
    k_l_table<<<(1 << 24) / 256, 256, 0, st>>>(ltab);
    return cudaGetLastError();
}

cudaError_t launch_target_lab(const uint8_t* rgb, int64_t n, double* lab, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_target_lab<<<blocks_for(n, 128), 128, 0, st>>>(rgb, n, lab);
    return cudaGetLastError();
}

cudaError_t launch_precision_probe(const TargetF32* tf, const TargetF64* td, int64_t n,
                                   const GridDev& g, const long long* qkey, float half_w,
                                   unsigned int* max_v_err_bits, unsigned int* max_lin_err_bits,
                                   unsigned int* max_lab_err_bits, unsigned long long* counts,
                                   int num_sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_precision_probe<<<num_sms * 8, 256, 0, st>>>(tf, td, n, g, qkey, half_w, max_v_err_bits,
                                                    max_lin_err_bits, max_lab_err_bits, counts);
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
