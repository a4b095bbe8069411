// cvs_internal.h - interface between the host API (cvs_api.cpp) and the
// kernels (cvs_kernels.cu) of libcvsearch.  Plain structs, no CUDA device code.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cvsearch.h"

namespace cvs {

// Per-target accumulator of the search (16 bytes): passing count, bits of the
// largest passing radius as float (-1.0f if none; non-negative floats order as
// integers), pattern bits, and one spare word.
struct __align__(16) Acc {
    int32_t count;
    int32_t rmax_bits;
    uint32_t pmask;
    uint32_t pad;
};

struct TargetF32;  // cvs_device.cuh
struct TargetF64;

// Grid tables on the device (owned by the context).
struct GridDev {
    int32_t K = 0, N = 0;      // radii, angles
    int32_t H = 0;             // angle slots per radius (N/2 when folded, else N)
    int32_t sym = 0;           // 1 if angles fold by +180 degrees
    int32_t arcs_ok = 0;       // folded and evenly spaced: slot h at angle th0 + h pi / H
    int32_t arcs = 0;          // the search walks per-radius angle ranges (arcs_ok and enabled)
    float th0 = 0.0f;          // angle of slot 0 (radians)
    float inv_step = 0.0f;     // slots per radian (H / pi)
    double rmax = 0.0;
    float* r32 = nullptr;      // K
    float2* sc32 = nullptr;    // N: (sin/500, -cos/200) in FP32
    double* r64 = nullptr;     // K
    double* s64 = nullptr;     // N
    double* c64 = nullptr;     // N
};

struct ImageDesc {             // device-side image table entry
    const uint8_t* rgb;
    int64_t pitch;
    int32_t width, height;
    int64_t first;             // index of the image's first pixel in the flat target list
    float* max_r;
    int32_t* count;
    uint8_t* pmask;
};

// Threads per block of the search kernel (its launch bound is compiled for it).
constexpr int kSearchBlock = 128;
// Largest radius for which the FP32 path's error has been measured to stay far
// inside its flag window; grids with a larger radius run in FP64.
constexpr double kFp32MaxRadius = 32.0;
// Largest radius accepted at all (keeps every FP32 code far below 2^22).
constexpr double kMaxRadius = 1000.0;

struct LaunchShape {
    int block = kSearchBlock;  // threads per block (64 or kSearchBlock)
    int blocks_per_sm = 0;     // 0: as many as fit
    int kchunk = 0;            // radii per work item (0: automatic)
};

// Device counters of a search: [0] work items taken, [1] flagged slots,
// [2] slots re-decided in FP64, [3] pairs written by the list compaction,
// [4] slots skipped as certainly out of gamut, [5] slots below the first
// radius where a pair may pass.  The kernels get counters + 1.
constexpr int kNumCounters = 6;

struct SearchArgs {
    const TargetF32* tf;
    const TargetF64* td;
    Acc* acc;
    int64_t n_targets;
    GridDev grid;
    const long long* qkey;     // 257 threshold keys
    int32_t hi_min, lo_max;
    uint32_t mask2;
    int32_t clip;
    float half_w;              // 0.5 - W
    int32_t prec;              // cvs_precision
    int32_t list_mode;         // 1: leave each work item's passing-slot bitmap and count
    uint32_t target_id;        // index of target 0 of the launch (list records)
    uint32_t* item_bits;       // list mode: item_words words per work item of the batch
    int32_t item_words;
    uint32_t* item_count;      // list mode: passing slots per work item
    int64_t item0;             // list mode: batch index of the launch's first work item
    const double* ltab;        // L* of all 2^24 colours when the luminance limit is on, else NULL
    double max_dl;             // the limit on |L*(plus) - L*(minus)| of an emitted pair
    unsigned long long* work_counter;
    unsigned long long* stats; // [0] flagged, [1] rechecked, [3] skipped, [4] pruned
    LaunchShape shape;
    int num_sms;
    uint2* arc_ranges;         // angle ranges per (target, radius) of a chunk (grid.arcs, FP32)
    int64_t arc_cap;           // entries of arc_ranges
    void* ev_ranges;           // host: a cudaEvent_t recorded after the first ranges pass, or NULL
    unsigned ev_flags;         // host: its record flags
};

// List mode: most slots (kchunk x H) of one work item, i.e. of a warp's
// passing-slot bitmap in shared memory.
constexpr int kListMaxSlots = 8192;
constexpr int kListMaxRadii = 256;  // and at most this many radii

// The records of a pair list from the search's per-item bitmaps (one batch).
struct EmitArgs {
    const TargetF32* tf;
    const TargetF64* td;
    int64_t n_targets;
    GridDev grid;
    const long long* qkey;
    int32_t hi_min, lo_max;
    uint32_t mask2;
    int32_t clip;
    float half_w;
    int32_t prec;
    int32_t kchunk;            // radii per work item, as in the search
    const uint32_t* item_bits; // item_words words per item
    int32_t item_words;
    const int64_t* item_base;  // records before each item within its tile of the scan
    const int64_t* tile_base;  // records before each tile (absolute)
    cvs_pair* out;             // the records, in (target, k, m) order
    int64_t out_cap;           // records `out` holds (the rest are not written)
    int64_t* offs;             // offs[t] = first record of target t, offs[n] = the end
    uint32_t target_id;        // index of target 0, for the records
};

// Entries of the angle-range scratch: targets are searched in chunks of
// kArcScratchEntries / K (8 bytes per (target, radius)).
constexpr int64_t kArcScratchEntries = int64_t(1) << 25;

// The multi-threshold search: up to kMaxThresholdSets sets in one pass.
constexpr int kMaxThresholdSets = 16;
struct MultiArgs {
    const TargetF32* tf;
    const TargetF64* td;
    const int32_t* order;      // K radius indices sorted by (radius value, index)
    Acc* acc;                  // n_targets * n_thr, index t * n_thr + s
    int64_t n_targets;
    GridDev grid;
    const long long* qkey;
    int32_t n_thr;
    int32_t hi_min[kMaxThresholdSets], lo_max[kMaxThresholdSets];
    uint32_t pmask_sets[8];    // [p]: bit s set if set s enables pattern p (1..7)
    int32_t all_patterns;      // 1 if every set enables all seven patterns
    int32_t hi_min_all;        // the smallest hi_min of the sets
    int32_t clip;              // shared by all sets
    const double* ltab;        // L* of all 2^24 colours when some set has a luminance limit
    uint32_t dl_free;          // sets without a luminance limit
    int64_t max_dl_bits[kMaxThresholdSets];  // bits of each limited set's max_dl (> 0)
    float half_w;
    int32_t prec;
    int32_t kchunk;
    unsigned long long* work_counter;
    unsigned long long* stats;
    int num_sms;
    // angle ranges of the union of the sets (FP32, gamut reject, a grid with
    // angle ranges), or NULL for the plain walk: per chunk of arc_cap / K
    // targets the range pass fills arc_ranges, then the search walks the lists
    uint2* arc_ranges;
    int64_t arc_cap;
    void* ev_ranges;           // host: a cudaEvent_t recorded after the first ranges pass, or NULL
    unsigned ev_flags;         // host: its record flags
};

// The embedding step: per pixel the first passing pair of the requested
// pattern in (radius value, radius index, angle index) order.
struct EmbedArgs {
    const TargetF32* tf;
    const TargetF64* td;
    int64_t n;                  // pixels (width * height)
    const uint8_t* rgb;         // the image (HWC bytes, row pitch)
    int64_t pitch;
    int32_t width, height;
    const uint8_t* pattern;     // requested pattern per pixel (row pitch), 1..7; else none
    int64_t pattern_pitch;
    uint8_t* frame_a;           // plus colours (HWC bytes, row pitch frame_pitch)
    uint8_t* frame_b;           // minus colours
    int64_t frame_pitch;
    uint32_t* choice;           // dense width*height: k | m << 16, or 0xFFFFFFFF; may be NULL
    GridDev grid;
    const int32_t* order;       // K radius indices sorted by (radius value, index)
    const long long* qkey;
    int32_t hi_min, lo_max;
    uint32_t mask2;
    int32_t clip;
    float half_w;
    int32_t prec;
    const double* ltab;         // luminance limit on: L* of all 2^24 colours, else NULL
    double max_dl;
    unsigned long long* work_counter;
    unsigned long long* stats;  // [0] flagged slots decided exactly, [1] slots re-decided in FP64
    int num_sms;
};

// The embedding table: per colour and pattern the first hit's key
// (rank << 16 | h; rank = position of the radius in the sorted order).
struct FirstHitArgs {
    const TargetF32* tf;
    const TargetF64* td;
    int64_t n_targets;
    GridDev grid;
    const int32_t* order;       // K radius indices sorted by (radius value, index)
    const long long* qkey;
    int32_t hi_min, lo_max;
    uint32_t mask2;
    int32_t clip;
    float half_w;
    int32_t prec;
    int32_t kchunk;             // ranks per work item
    const double* ltab;         // luminance limit on: L* of all 2^24 colours, else NULL
    double max_dl;
    uint32_t* key;              // n_targets * 7, pattern p at t * 7 + p - 1; 0xFFFFFFFF = none
    unsigned long long* work_counter;
    unsigned long long* stats;
    int num_sms;
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_trig_table(const double* angles_dev, int n, double* s64, double* c64,
                              float2* sc32, int* status, cudaStream_t st);
cudaError_t launch_setup_colors(const uint8_t* rgb, int64_t n, double rmax, TargetF32* tf,
                                TargetF64* td, Acc* acc, cudaStream_t st);
cudaError_t launch_setup_images(const ImageDesc* imgs, int n_imgs, int64_t total, double rmax,
                                TargetF32* tf, TargetF64* td, Acc* acc, cudaStream_t st);
cudaError_t launch_search(const SearchArgs& a, cudaStream_t st);
// Slot counts of the angle ranges of targets 0, stride, ..., (nt - 1) stride:
// counts[0] = slots the ranges list, counts[1] = slots of the radii a plain
// walk searches.
cudaError_t launch_arc_probe(const SearchArgs& a, int64_t nt, int64_t stride,
                             unsigned long long* counts, cudaStream_t st);
// The angle-range pass alone (k_arc_ranges) for the nt targets at a.tf, with
// a.hi_min and the patterns of a.mask2, into out (nt * K entries).
cudaError_t launch_arc_pass(const SearchArgs& a, int64_t nt, uint2* out, cudaStream_t st);
cudaError_t launch_finalize_colors(const Acc* acc, int64_t n, float* max_r, int32_t* count,
                                   uint8_t* pmask, cudaStream_t st);
cudaError_t launch_search_multi(const MultiArgs& a, cudaStream_t st);
int multi_max_chunk();  // largest radii per work item of the multi-threshold search
cudaError_t launch_embed(const EmbedArgs& a, cudaStream_t st);
cudaError_t launch_first_hits(const FirstHitArgs& a, cudaStream_t st);
// keys -> 16-byte table entries: the exact codes of each hit and its choice
cudaError_t launch_first_finalize(const FirstHitArgs& a, const uint32_t* keys, uint4* entry,
                                  cudaStream_t st);
cudaError_t launch_etab_gather(const uint4* entry, const uint8_t* rgb, int64_t pitch,
                               int32_t width, int32_t height, const uint8_t* pattern,
                               int64_t pattern_pitch, uint8_t* frame_a, uint8_t* frame_b,
                               int64_t frame_pitch, uint32_t* choice_out, cudaStream_t st);
cudaError_t launch_init_acc(Acc* acc, int64_t n, cudaStream_t st);
cudaError_t launch_finalize_images(const Acc* acc, const TargetF64* td, int64_t n,
                                   const ImageDesc* imgs, cudaStream_t st);
// Per-batch colour de-duplication of the image search (cvs_dedup.cu).
// mark: present[c] = 1 for every pixel colour c (the map is cleared first).
cudaError_t launch_dedup_mark(const ImageDesc* imgs, int n_imgs, int64_t total, uint8_t* present,
                              cudaStream_t st);
// scan: index[c] = rank of present colour c, unique_rgb = the present colours
// in colour order, *n_unique = their number; block_sums: 1024 ints of scratch.
cudaError_t launch_dedup_scan(const uint8_t* present, int* block_sums, int* n_unique,
                              int32_t* index, uint8_t* unique_rgb, cudaStream_t st);
// gather: every pixel's maps from acc[index[its colour]].
cudaError_t launch_dedup_gather(const ImageDesc* imgs, int n_imgs, int64_t total,
                                const int32_t* index, const Acc* acc, cudaStream_t st);
// L* of all 2^24 8-bit colours (index R << 16 | G << 8 | B), as step 1 forms it.
cudaError_t launch_l_table(double* ltab, cudaStream_t st);
cudaError_t launch_target_lab(const uint8_t* rgb, int64_t n, double* lab, cudaStream_t st);
// FP32 against FP64 over every (target, k, m) plus colour; counts[0..2] =
// wrong FP32 codes, wrong codes the search would not flag, values examined.
cudaError_t launch_precision_probe(const TargetF32* tf, const TargetF64* td, int64_t n,
                                   const GridDev& g, const long long* qkey, float half_w,
                                   unsigned int* max_v_err_bits, unsigned int* max_lin_err_bits,
                                   unsigned int* max_lab_err_bits, unsigned long long* counts,
                                   int num_sms, cudaStream_t st);
cudaError_t copy_qkeys_to(long long* dst, cudaStream_t st);
// Capacity table (all 2^24 colours).
constexpr int kGatherBlock = 256;
constexpr int kGatherMaxImages = 32;
struct GatherBatch {              // kernel parameter (by value)
    int n;
    int64_t block_first[kGatherMaxImages];
    ImageDesc img[kGatherMaxImages];
};
cudaError_t launch_rgb_iota(uint8_t* rgb, int64_t first, int64_t n, cudaStream_t st);
cudaError_t launch_lut_pack(const Acc* acc, int64_t n, uint64_t* entry, uint8_t* pmask,
                            cudaStream_t st);
cudaError_t launch_lut_gather_images(const GatherBatch& b, int64_t total_blocks,
                                     const uint64_t* entry, const uint8_t* pmask, cudaStream_t st);
cudaError_t launch_lut_gather_colors(const uint8_t* rgb, int64_t n, const uint64_t* entry,
                                     const uint8_t* pmask, float* max_r, int32_t* count,
                                     uint8_t* pm, cudaStream_t st);
// Sets the thread-local text returned by cvs_last_error().
void set_error_message(const char* msg);
// Radii per work item of the search when the caller fixes none: enough work
// items to spread n_targets over every SM, but at least two warp iterations.
int auto_kchunk(int num_sms, int64_t n_targets, int K, int H);
// 1 if a table of N sines and cosines is exactly antisymmetric under +180
// degrees (entry m + N/2 = -entry m), so slot m stands for angles m, m + N/2.
int fold_by_180(const double* s, const double* c, int N);
// Validate a threshold set and allocate, ahead of any search on the context,
// what it needs (the L* table of the luminance limit).
cvs_status prepare_thresholds(cvs_ctx* c, const cvs_thresholds* t);
size_t target_f32_size();
size_t target_f64_size();
int search_smem_bytes(const GridDev& g, int block, int list);
// Pair lists: scan of the items' record counts (count << sym) into within-tile
// bases and tile bases (tile: ceil(n_items / 4096) entries; carry: device,
// records before the batch), then the records.
cudaError_t launch_pair_scan(const uint32_t* count, int sym, int64_t n_items, int64_t* within,
                             int64_t* tile, const int64_t* carry, cudaStream_t st);
cudaError_t launch_emit_pairs(const EmitArgs& a, int num_sms, cudaStream_t st);
void chain_constants(float Ax[3], float Bz[3]);

}  // namespace cvs
