// cvs_multi.cu - the multi-threshold colour-pair search (sm_103a): every
// candidate decided against up to kMaxThresholdSets (V_th, R_novib, mask) sets
// in one pass (§3 Experiments, Table 1).
//
// The pair codes are formed once per slot (cvs_slot32.cuh).  The decision is
// bit-sliced over the sets: a shared table maps a channel's code difference
// |d| (0..255, 256 = out of range) to two 16-bit masks, the sets that call the
// channel high and those that call it low, so a slot costs three table reads
// whatever the number of sets.  Per lane, passes are counted in bytes (four
// sets per word) and patterns are OR-ed into one set mask per pattern.  A work
// item takes its radii in decreasing order, so a lane's first pass of a set is
// its largest passing radius for that set: it is recorded once, in shared
// memory, and the warp's maximum is taken at the end of the item.
// Flagged slots are marked in a per-lane bitmap; after each segment they are
// queued per warp and decided 32 at a time, one per lane (so the long exact
// path runs with full warps, seldom): bounds once, every set from them, FP64
// codes when some set stays open.
// On a grid with angle ranges (FP32, gamut reject) a fast-path target's item
// walks only the slots listed by the range pass run for the union of the sets
// (the smallest hi_min and every enabled pattern), a superset of the slots
// that pass any set.
#include <cuda_runtime.h>

#include "cvs_device.cuh"
#include "cvs_internal.h"
#include "cvs_slot32.cuh"

namespace cvs {

namespace {

constexpr int kMultiWords = 7;                  // flag words per lane per segment
constexpr int kMultiSegIters = 32 * kMultiWords;  // < 256: byte counters cannot overflow
static_assert(kMultiSegIters <= kArcMaskWords, "a segment's start mask must fit its buffer");
constexpr int kMultiMaxChunk = 8192;            // radii per work item
constexpr int kMultiQueue = 64;                 // flagged-slot queue entries per warp
// per warp in shared memory: flag words, largest radius per set, queue
constexpr int kMultiWarpWords = kMultiWords * 32 + kMaxThresholdSets * 32 + kMultiQueue;

// Table entry of |d| = i: bit s set if set s calls the channel high (i >= hi_min[s]),
// bit 16 + s if it calls it low (i <= lo_max[s]); i = 256 stands for out of range.
__device__ __forceinline__ void build_set_table(uint32_t* ts, const MultiArgs& A) {
    for (int i = threadIdx.x; i < 257; i += blockDim.x) {
        uint32_t e = 0;
        for (int s = 0; s < A.n_thr; ++s) {
            if (i <= 255 && i >= A.hi_min[s]) e |= 1u << s;
            if (i <= A.lo_max[s]) e |= 1u << (16 + s);
        }
        ts[i] = e;
    }
}

__device__ __forceinline__ uint32_t fold16(uint32_t x) { return (x | (x >> 16)) & 0xFFFFu; }

// Sets passing with channel table entries e[3] (high planes in the low half);
// hR/hG/hB receive the passing sets' high planes.  in_range: all codes in 0..255.
template <bool ALLMASK>
__device__ __forceinline__ uint32_t pass_sets(const uint32_t e[3], bool in_range, uint32_t setmask,
                                              const uint32_t* pmask_sets, uint32_t& hR,
                                              uint32_t& hG, uint32_t& hB) {
    const uint32_t valid = fold16(e[0]) & fold16(e[1]) & fold16(e[2]);
    uint32_t ok = valid & (e[0] | e[1] | e[2]) & setmask & (in_range ? 0xFFFFu : 0u);
    hR = e[0] & ok;
    hG = e[1] & ok;
    hB = e[2] & ok;
    if (!ALLMASK) {  // sets whose mask disallows the slot's pattern fail
        // with the planes masked by ok, a pattern's minterm is empty outside ok
        // (every pattern 1..7 has a high channel)
        uint32_t allowed = 0;
        allowed |= (~hR & ~hG & hB) & pmask_sets[1];
        allowed |= (~hR & hG & ~hB) & pmask_sets[2];
        allowed |= (~hR & hG & hB) & pmask_sets[3];
        allowed |= (hR & ~hG & ~hB) & pmask_sets[4];
        allowed |= (hR & ~hG & hB) & pmask_sets[5];
        allowed |= (hR & hG & ~hB) & pmask_sets[6];
        allowed |= (hR & hG & hB) & pmask_sets[7];
        ok = allowed;
        hR &= ok;
        hG &= ok;
        hB &= ok;
    }
    return ok;
}

// Sets whose luminance limit the pair with exact codes qp, qm meets: those
// without a limit, and those whose max_dl is at least the larger |L* - L| of
// the two emitted colours (non-negative doubles order as their bit patterns).
// Called only for slots that pass some set, so it stays out of the slot loop.
__device__ __noinline__ uint32_t dl_sets(const MultiArgs& A, double L, const int qp[3],
                                         const int qm[3]) {
    const int ip = (qp[0] << 16) | (qp[1] << 8) | qp[2];
    const int im = (qm[0] << 16) | (qm[1] << 8) | qm[2];
    const double d = fmax(fabs(__dsub_rn(__ldg(A.ltab + ip), L)),
                          fabs(__dsub_rn(__ldg(A.ltab + im), L)));
    const long long db = __double_as_longlong(d);
    uint32_t m = A.dl_free;
    for (int s = 0; s < A.n_thr; ++s)
        if (db <= A.max_dl_bits[s]) m |= 1u << s;
    return m;
}

// Per-lane tallies of one work item.
struct MultiTally {
    uint32_t c4[4];  // pass counts, byte b of word j = set 4 j + b
    uint32_t pm[8];  // pm[p]: sets with a pass of pattern p
    uint32_t cnt;    // lane s: set s's count so far (flushed bytes)
};

__device__ __forceinline__ void tally_patterns(MultiTally& m, uint32_t hR, uint32_t hG,
                                               uint32_t hB) {
    m.pm[1] |= ~hR & ~hG & hB;
    m.pm[2] |= ~hR & hG & ~hB;
    m.pm[3] |= ~hR & hG & hB;
    m.pm[4] |= hR & ~hG & ~hB;
    m.pm[5] |= hR & ~hG & hB;
    m.pm[6] |= hR & hG & ~hB;
    m.pm[7] |= hR & hG & hB;
}

// (all four words whatever the number of sets: branch-free measured 2% faster)
__device__ __forceinline__ void tally_counts(MultiTally& m, uint32_t ok) {
#pragma unroll
    for (int j = 0; j < 4; ++j) m.c4[j] += (((ok >> (4 * j)) & 15u) * 0x00204081u) & 0x01010101u;
}

// Byte counters -> lane s's 32-bit count of set s.
__device__ __forceinline__ void flush_counts(MultiTally& m, int NT) {
    const unsigned lane = lane_id();
    for (int s = 0; s < NT; ++s) {
        const uint32_t v = __reduce_add_sync(0xFFFFFFFFu, (m.c4[s >> 2] >> (8 * (s & 3))) & 255u);
        if ((int)lane == s) m.cnt += v;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) m.c4[j] = 0;
}

// Exact decision of one flagged slot against every set; passes go straight to
// the accumulators (rare).
template <int PREC, bool FAST, bool CLIP, bool ALLMASK, bool DL>
__device__ __forceinline__ void multi_flagged(const MultiArgs& A, const float2* r2s,
                                              const float4* sc4s, const uint32_t* ts,
                                              const TargetF32& T, const ChainF32& C,
                                              const TargetF64& D, int64_t t, int kk, int h,
                                              uint32_t setmask, unsigned long long& n_re) {
    const int NT = A.n_thr;
    const Intervals I = intervals32<FAST>(T, C, r2s[kk], sc4s[h], A.half_w, CLIP ? 1 : 0);
    bool certain_out = false, maybe_out = false;
    if (!CLIP) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            certain_out |= I.hi[j] < 0 || I.lo[j] > 255;
            maybe_out |= I.lo[j] < 0 || I.hi[j] > 255;
        }
    }
    if (certain_out) return;
    uint32_t e[3], unstable = 0, cinv = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int dmax = max(I.hi[c] - I.lo[3 + c], I.hi[3 + c] - I.lo[c]);
        const int dmin = max(0, max(I.lo[c] - I.hi[3 + c], I.lo[3 + c] - I.hi[c]));
        const uint32_t eL = ts[min(dmin, 256)], eH = ts[min(dmax, 256)];
        const uint32_t stable = ~fold16(eL ^ eH) & 0xFFFFu;
        cinv |= stable & ~fold16(eL);  // certainly neither high nor low: the set fails
        unstable |= ~stable;
        e[c] = eL;
    }
    uint32_t open = (maybe_out ? 0xFFFFu : unstable) & ~cinv & setmask;
    uint32_t hR, hG, hB, ok = 0;
    if (!open) ok = pass_sets<ALLMASK>(e, true, setmask & ~cinv, A.pmask_sets, hR, hG, hB);
    // some set's decision depends on a code the bounds leave open, or (under a
    // luminance limit) a set passes and the limit needs the exact codes: FP64
    if (open || (DL && ok)) {
        int qp[3], qm[3];
        pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + __ldg(A.order + kk)), __ldg(A.grid.s64 + h),
                     __ldg(A.grid.c64 + h), A.qkey, qp, qm);
        bool in_range = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (CLIP) {
                qp[c] = min(max(qp[c], 0), 255);
                qm[c] = min(max(qm[c], 0), 255);
            }
            in_range = in_range && qp[c] >= 0 && qp[c] <= 255 && qm[c] >= 0 && qm[c] <= 255;
            e[c] = ts[min(abs(qp[c] - qm[c]), 256)];
        }
        ok = pass_sets<ALLMASK>(e, in_range, setmask, A.pmask_sets, hR, hG, hB);
        if (DL && ok) ok &= dl_sets(A, D.L, qp, qm);
        ++n_re;
    }
    if (!ok) return;
    const int inc = A.grid.sym ? 2 : 1;
    const int r_bits = __float_as_int(r2s[kk].x);
    for (int s = 0; s < NT; ++s) {
        if (!((ok >> s) & 1u)) continue;
        const int p = (int)((((hR >> s) & 1u) << 2) | (((hG >> s) & 1u) << 1) | ((hB >> s) & 1u));
        Acc* ac = A.acc + t * NT + s;
        atomicAdd(&ac->count, inc);
        atomicMax(&ac->rmax_bits, r_bits);
        atomicOr(&ac->pmask, 1u << (p - 1));
    }
}

// Decide the first n (<= 32) queued flagged slots (rank | h << 16), one per lane.
template <int PREC, bool FAST, bool CLIP, bool ALLMASK, bool DL>
__device__ __forceinline__ void drain_multi(const MultiArgs& A, const float2* r2s,
                                            const float4* sc4s, const uint32_t* ts,
                                            const TargetF32& T, const ChainF32& C,
                                            const TargetF64& D, int64_t t, const uint32_t* pq,
                                            int n, uint32_t setmask, unsigned long long& n_re) {
    const unsigned lane = lane_id();
    if ((int)lane < n) {
        const uint32_t v = pq[lane];
        multi_flagged<PREC, FAST, CLIP, ALLMASK, DL>(A, r2s, sc4s, ts, T, C, D, t, (int)(v & 0xFFFFu),
                                                 (int)(v >> 16), setmask, n_re);
    }
}

// Item totals: lane s publishes set s (count, largest passing radius, patterns).
__device__ __forceinline__ void publish_item(const MultiArgs& A, const MultiTally& m,
                                             const float* rmx, int64_t t) {
    const unsigned lane = lane_id();
    const int NT = A.n_thr;
    const int inc = A.grid.sym ? 2 : 1;
    __syncwarp();
    uint32_t pmask = 0;
#pragma unroll
    for (int p = 1; p <= 7; ++p) {
        const uint32_t wp = __reduce_or_sync(0xFFFFFFFFu, m.pm[p]);
        if ((wp >> lane) & 1u) pmask |= 1u << (p - 1);
    }
    int rbits_mine = __float_as_int(-1.0f);
    for (int s = 0; s < NT; ++s) {
        const uint32_t b = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(rmx[s * 32 + lane]));
        if ((int)lane == s && b != 0u) rbits_mine = (int)b;
    }
    __syncwarp();
    if ((int)lane < NT && m.cnt) {
        Acc* ac = A.acc + t * NT + lane;
        atomicAdd(&ac->count, (int)m.cnt * inc);
        atomicMax(&ac->rmax_bits, rbits_mine);
        atomicOr(&ac->pmask, pmask);
    }
}

// Iterations [it, end) of a work item (lanes at slot (rank kk, angle h),
// radii decreasing); from it_pow on, every radius stays above the sRGB linear
// segment and the encode skips its select.  (Splitting the range at it_pow
// into two loops of one variant each, as k_search does, measured slower
// here: 26.5 against 23.7 ms for the 12 Table 1 sets on the cube.)  Flagged
// slots set their bits in `bits` (bit advances per iteration).
template <int PREC, bool FAST, bool CLIP, bool ALLMASK, bool DL>
__device__ __forceinline__ void multi_iters(const MultiArgs& A, const float2* r2s,
                                            const uint32_t* ts, const float4* sc4s,
                                            const PairsT& P, const PairsC& PC,
                                            const TargetF64& D, MultiTally& m, float* rmx,
                                            uint32_t setmask, int nslots, int kk1,
                                            int& it, int end, int& kk, int& h, uint32_t& bits,
                                            uint32_t& bit, uint32_t& seen, int it_pow) {
    const unsigned lane = lane_id();
    const int H = A.grid.H;
    const int q32 = 32 / H, r32 = 32 - q32 * H;
    for (; it < end; ++it, bit <<= 1) {
        const bool active = it * 32 + (int)lane < nslots;
        const int kq = active ? kk : kk1 - 1, hq = active ? h : 0;
        uint32_t ok = 0, hR = 0, hG = 0, hB = 0;
        bool skip = false;
        if (PREC == CVS_PREC_FP32_RECHECK) {
            const float2 r2 = r2s[kq];
            const float4 sc = sc4s[hq];
            const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y));
            const float2 w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
            float2 lin[3];
            lin32<FAST>(P, PC, u2, w2, lin);
            // gamut reject: a warp whose pairs all leave the gamut passes no set
            skip = !CLIP && __all_sync(0xFFFFFFFFu, !active || surely_out32(lin));
            if (!skip) {
                int yp[3], ym[3];
                bool flag;
                if (it >= it_pow) flag = encode32<false>(lin, A.half_w, yp, ym, nullptr);
                else flag = encode32<true>(lin, A.half_w, yp, ym, nullptr);
                flag = flag && active;
                if (flag) bits |= bit;
                uint32_t e[3];
                uint32_t o = 0;
                int qa[3], qb[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int a = yp[c] - kMagicBits, b = ym[c] - kMagicBits;
                    if (CLIP) {
                        a = min(max(a, 0), 255);
                        b = min(max(b, 0), 255);
                    }
                    qa[c] = a;
                    qb[c] = b;
                    o |= (uint32_t)a | (uint32_t)b;
                    e[c] = ts[min(abs(a - b), 256)];
                }
                if (active && !flag) {
                    ok = pass_sets<ALLMASK>(e, o <= 255u, setmask, A.pmask_sets, hR, hG, hB);
                    if (DL && ok) {  // the luminance limits, per set
                        ok &= dl_sets(A, D.L, qa, qb);
                        hR &= ok;
                        hG &= ok;
                        hB &= ok;
                    }
                }
            }
        } else if (active) {
            int qp[3], qm[3];
            pair_codes64(D.L, D.a, D.b, __ldg(A.grid.r64 + __ldg(A.order + kq)),
                         __ldg(A.grid.s64 + hq), __ldg(A.grid.c64 + hq), A.qkey, qp, qm);
            uint32_t e[3];
            bool in_range = true;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (CLIP) {
                    qp[c] = min(max(qp[c], 0), 255);
                    qm[c] = min(max(qm[c], 0), 255);
                }
                in_range = in_range && qp[c] >= 0 && qp[c] <= 255 && qm[c] >= 0 &&
                           qm[c] <= 255;
                e[c] = ts[min(abs(qp[c] - qm[c]), 256)];
            }
            ok = pass_sets<ALLMASK>(e, in_range, setmask, A.pmask_sets, hR, hG, hB);
            if (DL && ok) {
                ok &= dl_sets(A, D.L, qp, qm);
                hR &= ok;
                hG &= ok;
                hB &= ok;
            }
        }
        if (!skip) {
            tally_counts(m, ok);
            tally_patterns(m, hR, hG, hB);
            uint32_t fresh = ok & ~seen;  // radii decrease: the first pass is the largest
            if (fresh) {
                seen |= fresh;
                const float r = r2s[kq].x;
                while (fresh) {
                    const int s = __ffs(fresh) - 1;
                    fresh &= fresh - 1u;
                    rmx[s * 32 + lane] = r;
                }
            }
        }
        h += r32;
        kk -= q32;
        const bool wrap = h >= H;
        h = wrap ? h - H : h;
        kk = wrap ? kk - 1 : kk;
    }
}

// One work item: target t, radius ranks [kk0, kk1), taken in decreasing order.
template <int PREC, bool FAST, bool CLIP, bool ALLMASK, bool DL>
__device__ __forceinline__ void multi_item(const MultiArgs& A, const float2* r2s,
                                           const float4* sc4s, const uint32_t* ts, uint32_t* fb,
                                           float* rmx, uint32_t* pq, const TargetF32& T,
                                           const ChainF32& C,
                                           const PairsC& PC, int64_t t, int kk0, int kk1,
                                           unsigned long long& n_flag,
                                           unsigned long long& n_re) {
    const unsigned lane = lane_id();
    const int H = A.grid.H, NT = A.n_thr;
    const uint32_t setmask = (1u << NT) - 1u;
    const TargetF64 D = A.td[t];
    const PairsT P = make_pairs(T);
    MultiTally m;
#pragma unroll
    for (int j = 0; j < 4; ++j) m.c4[j] = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) m.pm[p] = 0;
    m.cnt = 0;
    uint32_t seen = 0;  // sets this lane has seen pass (its largest radius is recorded)
    int pq_n = 0;       // queued flagged slots (warp-uniform)
    for (int s = 0; s < NT; ++s) rmx[s * 32 + lane] = 0.0f;  // radius 0 never passes
    // slot i of the item is (rank kk1 - 1 - i / H, i % H); lanes step by 32
    int kk = kk1 - 1 - (int)lane / H, h = (int)lane % H;
    int klo = kk0;      // ranks below klo certainly fail for every set
    int it_pow = 1 << 30;  // iterations from here on never reach the sRGB linear segment
    if (PREC == CVS_PREC_FP32_RECHECK && FAST) {
        klo = first_possible_radius(T, C, r2s, kk0, kk1, A.hi_min_all);
        const int k_split = first_linseg_radius(T, C, r2s, kk0, kk1);  // ranks below: pow only
        it_pow = ((kk1 - k_split) * H + 31) >> 5;
    }
    const int nslots = (kk1 - klo) * H;
    const int nit = (nslots + 31) >> 5;
    for (int seg0 = 0; seg0 < nit; seg0 += kMultiSegIters) {
        const int seg1 = min(seg0 + kMultiSegIters, nit);
        for (int w = 0, it = seg0; it < seg1; ++w) {
            uint32_t bits = 0;
            const int wend = min(seg1, it + 32);
            uint32_t bit = 1u;
            multi_iters<PREC, FAST, CLIP, ALLMASK, DL>(A, r2s, ts, sc4s, P, PC, D, m, rmx, setmask,
                                                       nslots, kk1, it, wend, kk, h, bits, bit,
                                                       seen, it_pow);
            if (PREC == CVS_PREC_FP32_RECHECK) fb[w * 32 + lane] = bits;
        }
        flush_counts(m, NT);
        if (PREC == CVS_PREC_FP32_RECHECK) {  // queue the segment's flagged slots
            __syncwarp();
            const int nwords = (seg1 - seg0 + 31) >> 5;
            for (int w = 0; w < nwords; ++w) {
                uint32_t bits = fb[w * 32 + lane];
                while (true) {
                    const bool has = bits != 0u;
                    const unsigned ball = __ballot_sync(0xFFFFFFFFu, has);
                    if (!ball) break;
                    if (has) {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        const int i = (seg0 + 32 * w + j) * 32 + (int)lane;
                        const int dk = i / H;
                        pq[pq_n + __popc(ball & ((1u << lane) - 1u))] =
                            (uint32_t)(kk1 - 1 - dk) | ((uint32_t)(i - dk * H) << 16);
                        ++n_flag;
                    }
                    pq_n += __popc(ball);  // below kMultiQueue: at most 31 + 32
                    __syncwarp();
                    if (pq_n >= 32) {
                        drain_multi<PREC, FAST, CLIP, ALLMASK, DL>(A, r2s, sc4s, ts, T, C, D, t, pq,
                                                               32, setmask, n_re);
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
    }
    if (PREC == CVS_PREC_FP32_RECHECK && pq_n > 0)
        drain_multi<PREC, FAST, CLIP, ALLMASK, DL>(A, r2s, sc4s, ts, T, C, D, t, pq, pq_n, setmask,
                                               n_re);
    publish_item(A, m, rmx, t);
}

// Steps [b, bend) of a list walk (lane at position b + lane of the list in
// al, whose start mask covers the segment from seg; positions from pend on
// inactive): as multi_iters, in the chain variant FAST, with each lane's
// (rank, angle) from its list entry.  The encode keeps the
// sRGB linear-segment select throughout: the loop body stays one variant (a
// choice per step, or two loops split at the last radius that may reach the
// segment, measured 2.5% and 6% slower: the kernel waits on instruction
// fetch, and both make the loop longer).
template <bool FAST, bool ALLMASK, bool DL>
__device__ __forceinline__ void multi_list_iters(const MultiArgs& A, const float2* r2s,
                                                 const uint32_t* ts, const float4* sc4s,
                                                 const PairsT& P, const PairsC& PC,
                                                 const TargetF64& D, MultiTally& m, float* rmx,
                                                 uint32_t setmask, const uint32_t* al,
                                                 int kb, int pend, int seg, int& b,
                                                 int bend, int& j0, uint32_t& bits,
                                                 uint32_t& seen) {
    const unsigned lane = lane_id();
    const uint32_t* msk = al + 2 * kArcEntries;
    uint32_t bit = 1u;
    for (; b < bend; b += 32, bit <<= 1) {
        const int p = b + (int)lane;
        const bool active = p < pend;
        const uint32_t e = list_step(al, msk[(b - seg) >> 5], j0);
        const int kq = active ? kb + (int)(e & 127u) : kb;
        const int hq = active ? p + (int)(e >> 8) - kArcBias : 0;
        const float2 r2 = r2s[kq];
        const float4 sc = sc4s[hq];
        const float2 u2 = __fmul2_rn(r2, f2(sc.x, sc.y));
        const float2 w2 = __fmul2_rn(r2, f2(sc.z, sc.w));
        float2 lin[3];
        lin32<FAST>(P, PC, u2, w2, lin);
        // gamut reject: a warp whose pairs all leave the gamut passes no set
        if (__all_sync(0xFFFFFFFFu, !active || surely_out32(lin))) continue;
        int yp[3], ym[3];
        bool flag;
        flag = encode32<true>(lin, A.half_w, yp, ym, nullptr);
        flag = flag && active;
        if (flag) bits |= bit;
        uint32_t e3[3];
        uint32_t o = 0;
        int qa[3], qb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int a = yp[c] - kMagicBits, bq = ym[c] - kMagicBits;
            qa[c] = a;
            qb[c] = bq;
            o |= (uint32_t)a | (uint32_t)bq;
            e3[c] = ts[min(abs(a - bq), 256)];
        }
        uint32_t ok = 0, hR = 0, hG = 0, hB = 0;
        if (active && !flag) {
            ok = pass_sets<ALLMASK>(e3, o <= 255u, setmask, A.pmask_sets, hR, hG, hB);
            if (DL && ok) {  // the luminance limits, per set
                ok &= dl_sets(A, D.L, qa, qb);
                hR &= ok;
                hG &= ok;
                hB &= ok;
            }
        }
        tally_counts(m, ok);
        tally_patterns(m, hR, hG, hB);
        uint32_t fresh = ok & ~seen;  // ranks decrease along a lane: the first pass is the largest
        if (fresh) {
            seen |= fresh;
            const float r = r2.x;
            while (fresh) {
                const int s = __ffs(fresh) - 1;
                fresh &= fresh - 1u;
                rmx[s * 32 + lane] = r;
            }
        }
    }
}

// A work item (FP32, gamut reject) on a grid with angle ranges: the listed
// slots of ranks [kk0, kk1), of the fast-path radii (FAST) or of the
// slow-path ones, in blocks of kArcRadii from the top, each block's
// ranges listed in decreasing rank (so that a lane meets its radii in
// decreasing order, as in multi_item) and walked 32 positions a step; flagged
// slots are found again in the list and queued as in multi_item.
template <bool FAST, bool ALLMASK, bool DL>
__device__ __forceinline__ void multi_item_arcs(const MultiArgs& A, const float2* r2s,
                                                const float4* sc4s, const uint32_t* ts,
                                                uint32_t* fb, float* rmx, uint32_t* pq,
                                                uint32_t* al, const TargetF32& T,
                                                const ChainF32& C, const PairsC& PC, int64_t t,
                                                int kk0, int kk1, unsigned long long& n_flag,
                                                unsigned long long& n_re) {
    constexpr int PREC = CVS_PREC_FP32_RECHECK;
    const unsigned lane = lane_id();
    const int K = A.grid.K, NT = A.n_thr;
    const uint32_t setmask = (1u << NT) - 1u;
    const TargetF64 D = A.td[t];
    const PairsT P = make_pairs(T);
    MultiTally m;
#pragma unroll
    for (int j = 0; j < 4; ++j) m.c4[j] = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) m.pm[p] = 0;
    m.cnt = 0;
    uint32_t seen = 0;
    int pq_n = 0;
    for (int s = 0; s < NT; ++s) rmx[s * 32 + lane] = 0.0f;
    uint32_t* pos = al + kArcEntries;
    const uint2* ranges = A.arc_ranges + t * K;
    for (int kb1 = kk1; kb1 > kk0; kb1 -= kArcRadii) {
        const int kb = max(kk0, kb1 - kArcRadii);
        int nf = 0, pf = 0;  // the list's entries and positions
        for (int kg = kb1 - 1; kg >= kb; kg -= 32) {
            const int kk = kg - (int)lane;
            uint2 o = kk >= kb ? __ldg(ranges + __ldg(A.order + kk)) : make_uint2(0u, 0u);
            if (((o.x & kSlowRadius) != 0u) == FAST) o = make_uint2(0u, 0u);  // the other walk's
            o.x &= ~kSlowRadius;
            const uint32_t w0 = o.x, w1 = o.y;
            const int l0 = (int)(w0 >> 16), l1 = (int)(w1 >> 16);
            const int n = (l0 > 0 ? 1 : 0) + (l1 > 0 ? 1 : 0);
            int nr, pr;
            const int eoff = nf + warp_exclusive_sum(n, nr);
            const int poff = pf + warp_exclusive_sum(l0 + l1, pr);
            const uint32_t koff = (uint32_t)(kk - kb);
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
        if (lane == 0) pos[nf] = (uint32_t)pf;
        __syncwarp();
        int j0 = -1;
        for (int seg = 0; seg < pf; seg += 32 * kMultiSegIters) {
            const int seg_end = min(pf, seg + 32 * kMultiSegIters);
            list_mask(al, nf, seg, (seg_end - seg + 31) >> 5, j0);
            int b = seg;
            for (int w = 0; b < seg_end; ++w) {
                uint32_t bits = 0;
                multi_list_iters<FAST, ALLMASK, DL>(A, r2s, ts, sc4s, P, PC, D, m, rmx, setmask, al,
                                              kb, pf, seg, b, min(seg_end, b + 32 * 32), j0,
                                              bits, seen);
                fb[w * 32 + lane] = bits;
            }
            flush_counts(m, NT);
            __syncwarp();
            // queue the segment's flagged slots
            const int nwords = (((seg_end - seg + 31) >> 5) + 31) >> 5;
            for (int w = 0; w < nwords; ++w) {
                uint32_t bits = fb[w * 32 + lane];
                while (true) {
                    const bool has = bits != 0u;
                    const unsigned ball = __ballot_sync(0xFFFFFFFFu, has);
                    if (!ball) break;
                    if (has) {
                        const int i = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        const int p = seg + 32 * (32 * w + i) + (int)lane;
                        const uint32_t e = list_entry(al, 0, nf, p);
                        const uint32_t kk = (uint32_t)kb + (e & 127u);
                        const uint32_t h = (uint32_t)(p + (int)(e >> 8) - kArcBias);
                        pq[pq_n + __popc(ball & ((1u << lane) - 1u))] = kk | (h << 16);
                        ++n_flag;
                    }
                    pq_n += __popc(ball);  // below kMultiQueue: at most 31 + 32
                    __syncwarp();
                    if (pq_n >= 32) {
                        drain_multi<PREC, FAST, false, ALLMASK, DL>(A, r2s, sc4s, ts, T, C, D, t,
                                                                    pq, 32, setmask, n_re);
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
        __syncwarp();  // the list is rebuilt for the next block of radii
    }
    if (pq_n > 0)
        drain_multi<PREC, FAST, false, ALLMASK, DL>(A, r2s, sc4s, ts, T, C, D, t, pq, pq_n, setmask,
                                                    n_re);
    publish_item(A, m, rmx, t);
}

// ARCS (FP32, gamut reject, a grid with angle ranges): 1 = the range walk of
// every target's fast-path radii, 2 = that of the slow-path radii of the
// targets that have some (a second launch, with the slow chain); 0 = the plain
// walk.  One chain variant per kernel: walking both in one kernel measured 13%
// slower (17.5 against 15.3 ms for the 12 Table 1 sets on the cube), as the
// kernel waits on instruction fetch and two walks at once double its hot code.
template <int PREC, bool CLIP, bool ALLMASK, bool DL, int ARCS>
__global__ void __launch_bounds__(kSearchBlock) k_search_multi(const MultiArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = A.grid.K, H = A.grid.H;
    float2* r2s = reinterpret_cast<float2*>(smem);
    float4* sc4s = reinterpret_cast<float4*>(smem + ((K * 8 + 15) & ~15));
    uint32_t* ts = reinterpret_cast<uint32_t*>(smem + ((K * 8 + 15) & ~15) + H * 16);
    uint32_t* per_warp = ts + 260;  // 257 table entries, padded to 16 bytes
    const int warp = threadIdx.x >> 5;
    uint32_t* fb = per_warp + warp * kMultiWarpWords;
    float* rmx = reinterpret_cast<float*>(fb + kMultiWords * 32);
    uint32_t* pq = fb + kMultiWords * 32 + kMaxThresholdSets * 32;
    uint32_t* al = ARCS ? per_warp + (blockDim.x >> 5) * kMultiWarpWords + warp * kArcWords
                        : nullptr;
    build_set_table(ts, A);
    for (int i = threadIdx.x; i < K; i += blockDim.x) r2s[i] = dup(A.grid.r32[A.order[i]]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        const float2 sc = A.grid.sc32[i];
        sc4s[i] = make_float4(sc.x, -sc.x, sc.y, -sc.y);
    }
    const unsigned lane = lane_id();
    for (int i = (int)lane; i < kMultiWords * 32; i += 32) fb[i] = 0u;
    __syncthreads();
    ChainF32 C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C.Ax[c] = __double2float_rn(__dmul_rn(c_MI[3 * c], c_W[0]));
        C.Bz[c] = __double2float_rn(__dmul_rn(c_MI[3 * c + 2], c_W[2]));
    }
    const PairsC PC = make_pairs(C);
    unsigned long long n_flag = 0, n_re = 0;
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
        const int k0 = kc * kchunk, k1 = min(k0 + kchunk, K);
        TargetF32 T{};
        if (PREC == CVS_PREC_FP32_RECHECK) T = A.tf[t];
        if (ARCS == 1) {
            multi_item_arcs<true, ALLMASK, DL>(A, r2s, sc4s, ts, fb, rmx, pq, al, T, C, PC, t, k0,
                                               k1, n_flag, n_re);
        } else if (ARCS == 2) {  // a fast-path target has no slow-path radius
            if (!(T.flags & 1u))
                multi_item_arcs<false, ALLMASK, DL>(A, r2s, sc4s, ts, fb, rmx, pq, al, T, C, PC, t,
                                                    k0, k1, n_flag, n_re);
        } else if (PREC == CVS_PREC_FP32_RECHECK && (T.flags & 1u)) {
            multi_item<PREC, true, CLIP, ALLMASK, DL>(A, r2s, sc4s, ts, fb, rmx, pq, T, C, PC, t,
                                                  k0, k1, n_flag, n_re);
        } else {
            multi_item<PREC, false, CLIP, ALLMASK, DL>(A, r2s, sc4s, ts, fb, rmx, pq, T, C, PC, t,
                                                   k0, k1, n_flag, n_re);
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

int multi_smem_bytes(const GridDev& g, int block, bool arcs) {
    return ((g.K * 8 + 15) & ~15) + g.H * 16 + 260 * 4 +
           (block / 32) * (kMultiWarpWords + (arcs ? kArcWords : 0)) * 4;
}

template <int PREC, bool CLIP, bool ALLMASK, bool DL>
cudaError_t launch_multi_t(const MultiArgs& a, cudaStream_t st) {
    const int block = kSearchBlock;
    constexpr bool kArcsKernel = PREC == CVS_PREC_FP32_RECHECK && !CLIP;
    const bool arcs = kArcsKernel && a.arc_ranges && a.arc_cap >= a.grid.K;
    const int smem = multi_smem_bytes(a.grid, block, arcs);
    const void* fn = arcs ? (const void*)k_search_multi<PREC, CLIP, ALLMASK, DL, kArcsKernel>
                          : (const void*)k_search_multi<PREC, CLIP, ALLMASK, DL, 0>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (!arcs) {
        k_search_multi<PREC, CLIP, ALLMASK, DL, 0><<<a.num_sms * per_sm, block, smem, st>>>(a);
        return cudaGetLastError();
    }
    // the range walk of the slow-path radii (slow chain), launched after each chunk's
    const void* fn_slow = (const void*)k_search_multi<PREC, CLIP, ALLMASK, DL, kArcsKernel ? 2 : 0>;
    e = cudaFuncSetAttribute(fn_slow, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm_slow = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_slow, fn_slow, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm_slow < 1) per_sm_slow = 1;
    // per chunk of targets: the range pass for the union of the sets (the
    // smallest hi_min, every enabled pattern), then the search
    SearchArgs pass{};
    pass.grid = a.grid;
    pass.hi_min = a.hi_min_all;
    for (int p = 1; p <= 7; ++p)
        if (a.pmask_sets[p]) pass.mask2 |= 1u << p;
    pass.num_sms = a.num_sms;
    const int64_t chunk = a.arc_cap / a.grid.K;
    for (int64_t t0 = 0; t0 < a.n_targets; t0 += chunk) {
        const int64_t nt = a.n_targets - t0 < chunk ? a.n_targets - t0 : chunk;
        MultiArgs c = a;
        c.tf += t0;
        c.td += t0;
        c.acc += t0 * a.n_thr;
        c.n_targets = nt;
        if (t0 > 0) {
            e = cudaMemsetAsync(c.work_counter, 0, sizeof(unsigned long long), st);
            if (e != cudaSuccess) return e;
        }
        pass.tf = c.tf;
        e = launch_arc_pass(pass, nt, a.arc_ranges, st);
        if (e != cudaSuccess) return e;
        if (t0 == 0 && a.ev_ranges) {
            e = cudaEventRecordWithFlags((cudaEvent_t)a.ev_ranges, st, a.ev_flags);
            if (e != cudaSuccess) return e;
        }
        k_search_multi<PREC, CLIP, ALLMASK, DL, kArcsKernel><<<a.num_sms * per_sm, block, smem, st>>>(
            c);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c.work_counter, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        k_search_multi<PREC, CLIP, ALLMASK, DL, kArcsKernel ? 2 : 0>
            <<<a.num_sms * per_sm_slow, block, smem, st>>>(c);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int PREC, bool DL>
cudaError_t launch_multi_d(const MultiArgs& a, cudaStream_t st) {
    if (a.clip)
        return a.all_patterns ? launch_multi_t<PREC, true, true, DL>(a, st)
                              : launch_multi_t<PREC, true, false, DL>(a, st);
    return a.all_patterns ? launch_multi_t<PREC, false, true, DL>(a, st)
                          : launch_multi_t<PREC, false, false, DL>(a, st);
}

// DL: some set carries a luminance limit (a separate instantiation, so that
// the sets without one run the loop without it)
template <int PREC>
cudaError_t launch_multi_p(const MultiArgs& a, cudaStream_t st) {
    return a.ltab ? launch_multi_d<PREC, true>(a, st) : launch_multi_d<PREC, false>(a, st);
}

}  // namespace

int multi_max_chunk() { return kMultiMaxChunk; }

cudaError_t launch_search_multi(const MultiArgs& a, cudaStream_t st) {
    if (a.kchunk < 1 || a.kchunk > kMultiMaxChunk || a.n_thr < 1 || a.n_thr > kMaxThresholdSets)
        return cudaErrorInvalidValue;
    return a.prec == CVS_PREC_FP64 ? launch_multi_p<CVS_PREC_FP64>(a, st)
                                   : launch_multi_p<CVS_PREC_FP32_RECHECK>(a, st);
}

cudaError_t launch_init_acc(Acc* acc, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_init_acc<<<(int)((n + 255) / 256), 256, 0, st>>>(acc, n);
    return cudaGetLastError();
}

}  // namespace cvs
