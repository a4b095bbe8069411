/*
 * cvsearch.h - C ABI of libcvsearch, a GB300 (sm_103a) implementation of the
 * colour-pair search of "Accelerated and Optimized Search of Imperceptible
 * Color Vibration for Embedding Information into LCD images" (Hattori and
 * Hiraki, SIGGRAPH Asia 2022 Posters).
 *
 * The operation (paper §2 Methods, Fig. 1b and Fig. 2; §3 Experiments and
 * Table 1):
 *   For a target colour, take its CIE L*a*b* coordinates (L, a, b).  For every
 *   radius i = radii[k] and angle j = angles_deg[m] form the point-symmetric
 *   pair
 *       plus  = (L, a + i sin j, b + i cos j)      ("D_a", "D_b" added)
 *       minus = (L, a - i sin j, b - i cos j)      (subtracted)
 *   at fixed L* (the colour-vibration condition), convert both back to 8-bit
 *   sRGB and keep the pair if, in every RGB channel, the difference
 *   |plus_c - minus_c| is either "high" (> V_th) or "low" (< V_th * R_novib),
 *   the high/low word (R,G,B) = p is not 000, and p is enabled in the pattern
 *   mask (the embedding-signal condition; patterns 100 ... 111 of Table 1).
 *
 * Number semantics (where the paper is silent):
 *   - sRGB IEC 61966-2-1, D65 white, CIE 1976 L*a*b*; FP64 in the order of the
 *     textbook formulas; the target's cube roots are correctly rounded.
 *   - sin j / cos j are the correctly rounded values of the exact angle in
 *     degrees, so angle j + 180 gives exactly the swapped pair.
 *   - 8-bit code = floor(255 * enc(lin) + 1/2) of the FP64 linear value, in
 *     exact arithmetic.  Gamut: mode 0 rejects a pair with any code outside
 *     [0, 255]; mode 1 clamps the codes.
 *   The results are identical to those of a plain FP64 evaluation in that
 *   order: the FP32 fast path re-decides in FP64 every candidate whose FP32
 *   codes could be wrong.
 *
 * Threading: a cvs_ctx may be used by one host thread at a time.  Its
 * scratch memory is shared by its calls, so asynchronous calls on one context
 * must be issued on one stream (or the caller synchronises between streams);
 * a call with a different grid waits for the device before replacing tables.
 * Memory: the caller owns every input and output buffer; the context owns its
 * scratch memory (tables, per-target constants, work counters) and frees it
 * in cvs_destroy.
 * Errors: every entry point returns a cvs_status; cvs_last_error() gives a
 * thread-local message for the last failure.  Invalid arguments are reported
 * before any device work is issued.  Asynchronous entry points report CUDA
 * launch errors immediately and execution errors at the next synchronising
 * call (cvs_synchronize or a synchronous entry point).
 */
#ifndef CVSEARCH_H
#define CVSEARCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CVS_OK = 0,
    CVS_ERR_INVALID_ARG = 1, /* bad pointer, size, NaN, out-of-range parameter */
    CVS_ERR_NO_MEMORY = 2,   /* device or pinned host allocation failed */
    CVS_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    CVS_ERR_TRUNCATED = 4,   /* output capacity too small; *n_out = required count */
    CVS_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
    CVS_ERR_NUMERIC = 6      /* a table value could not be certified (never seen) */
} cvs_status;

/* Arithmetic of a search.  Both give identical results.  FP32_RECHECK runs
 * the bulk in FP32 and re-decides in FP64 every candidate whose FP32 codes
 * could be wrong; its error bound is validated for radii up to 32 (over all
 * 2^24 colours), so on a grid with a larger radius an FP32_RECHECK call
 * returns CVS_ERR_INVALID_ARG, unless option "fp64_fallback" is 1, in which
 * case it runs in FP64 (about 100x slower; cvs_stats.precision says which
 * ran). */
typedef enum {
    CVS_PREC_FP32_RECHECK = 0, /* FP32 bulk, FP64 re-decision near rounding boundaries */
    CVS_PREC_FP64 = 1          /* every candidate in FP64 (comparison form) */
} cvs_precision;

typedef struct cvs_ctx cvs_ctx;

/* The (radius i, angle j) grid of §2 Methods.  Host pointers, read during the
 * call.  radii: in [0, 1000] L*a*b* units, at most 8192 values.
 * angles_deg: finite, in degrees, at most 8192 values.  When the angle list
 * is closed under +180 degrees with angles_deg[m + n/2] = angles_deg[m] + 180
 * (mod 360), each symmetric pair is evaluated once. */
typedef struct {
    const double* radii;
    int32_t n_radii;
    const double* angles_deg;
    int32_t n_angles;
} cvs_grid;

/* Conditions a pair must meet: the embedding-signal condition (§3
 * Experiments, Table 1), the gamut, and an optional refinement of the
 * colour-vibration condition (§2 Methods).  32 bytes.
 * v_th: finite, >= 0.  r_novib: in (0, 1].  A channel difference d is high
 * if d > v_th and low if d < v_th * r_novib (exact comparisons).
 * pattern_mask: bit p-1 enables pattern p = (hi_R << 2) | (hi_G << 1) | hi_B,
 * p = 1..7 (0x7F = all seven patterns of Table 1).
 * gamut_mode: 0 = reject pairs with a code outside [0,255], 1 = clamp.
 * max_dl: luminance limit on the emitted pair.  §2 Methods keeps L* fixed
 *   before quantisation and states no tolerance after it; with a positive,
 *   finite max_dl a passing pair is kept only if each of its two emitted
 *   8-bit colours has an L* (step 1 of §2 Methods applied to its codes,
 *   clamped in clip mode) within max_dl of the target's L*.  0 (what a
 *   zero-initialised struct holds) and +inf mean no limit; a negative value
 *   or NaN is CVS_ERR_INVALID_ARG.  The first call on a context with a limit
 *   builds a table of the L* of all 2^24 colours (128 MiB, synchronous). */
typedef struct {
    double v_th;
    double r_novib;
    uint32_t pattern_mask;
    int32_t gamut_mode;
    double max_dl;
} cvs_thresholds;

/* One passing candidate (16 bytes).  k, m: radius and angle indices;
 * plus / minus: the 8-bit sRGB of the two colours; pattern: 1..7;
 * flags: bit 0 = the codes were computed in FP64 (some FP32 code lay within
 * the window of a rounding boundary, or the call ran in FP64); target:
 * caller's index. */
typedef struct {
    uint16_t k, m;
    uint8_t plus[3], minus[3];
    uint8_t pattern, flags;
    uint32_t target;
} cvs_pair;

/* Per-target results (Table 2's question, per colour or pixel), device
 * pointers to n entries each, written by the search:
 *   max_r: largest radius of a passing candidate, -1.0f if none;
 *   count: number of passing (k, m) candidates;
 *   pmask: bit p-1 set if some passing candidate carries pattern p. */
typedef struct {
    float* max_r;
    int32_t* count;
    uint8_t* pmask;
} cvs_capacity_map;

/* An 8-bit sRGB image, HWC (R, G, B bytes per pixel), device pointer.
 * Row y starts at rgb + y * pitch_bytes; pitch_bytes >= 3 * width. */
typedef struct {
    const uint8_t* rgb;
    int32_t width;
    int32_t height;
    int64_t pitch_bytes;
} cvs_image;

/* Counters of the last search call on a context (filled when the call has
 * completed, i.e. after cvs_synchronize for asynchronous calls). */
typedef struct {
    int64_t candidates;      /* (target, k, m) candidates decided */
    int64_t colors_fp32;     /* colour conversions done in FP32 */
    int64_t flagged;         /* candidates with a code within the FP32 window */
    int64_t rechecked;       /* candidates re-decided in FP64 */
    int64_t targets;         /* targets (colours or pixels) searched */
    int32_t symmetric;       /* 1 if the angle list was folded by +180 degrees */
    int32_t precision;       /* cvs_precision of the call */
    double search_ms;        /* device time of the search kernel (CUDA events on the
                                call's stream) */
    int64_t skipped;         /* candidates rejected without encoding: in gamut-reject
                                mode, a warp's 32 slots whose linear RGB all lie
                                certainly outside the range of codes 0..255 */
    int64_t pruned;          /* candidates rejected without any work: radii below the
                                first one where, by a bound on the pair's code
                                difference, some channel could be high, and (option
                                "angle_ranges") slots outside a radius's ranges */
    double ranges_ms;        /* of search_ms, the angle-ranges pass before the search
                                kernel (first chunk of targets; 0 without it) */
} cvs_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (the device is made current for
 * every call on the context).  *ctx receives the handle, owned by the caller
 * and released with cvs_destroy.  mem_budget_bytes caps the device memory the
 * context itself allocates (its scratch and tables, including temporary
 * buffers of a table build; not the tables returned by cvs_lut_build and
 * cvs_etab_build, which belong to the caller): a call that would exceed it
 * returns CVS_ERR_NO_MEMORY before any device work, and the context stays
 * usable.  0 = no cap.  Returns CVS_ERR_CUDA if the device is not usable. */
cvs_status cvs_create(cvs_ctx** ctx, int device, size_t mem_budget_bytes);

/* Free the context and all scratch memory it owns (waits for its work). */
void cvs_destroy(cvs_ctx* ctx);

/* Thread-local text of the last error, or "" (never NULL). */
const char* cvs_last_error(void);

/* Library version as "major.minor.patch". */
const char* cvs_version(void);

/* Resolve the embedding-signal thresholds (§3 Experiments) to integer bounds
 * on the channel difference d in [0, 255]: high iff d >= *hi_min, low iff
 * d <= *lo_max.  Host only; no device work.  Validates *thr. */
cvs_status cvs_signal_bounds(const cvs_thresholds* thr, int32_t* hi_min, int32_t* lo_max);

/* Correctly rounded sin / cos of the angles in degrees as the search uses
 * them (§2 Methods: D_a = i sin j, D_b = i cos j), computed on the device.
 * angles_deg: host, n values; sin_out / cos_out: host, n doubles each.
 * Synchronous. */
cvs_status cvs_trig_table(cvs_ctx* ctx, const double* angles_deg, int32_t n,
                          double* sin_out, double* cos_out);

/* L*a*b* of n 8-bit sRGB colours (step 1 of §2 Methods) on the device.
 * rgb_dev: device, 3n bytes; lab_dev: device, 3n doubles (L, a, b).
 * Asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream). */
cvs_status cvs_target_lab(cvs_ctx* ctx, const uint8_t* rgb_dev, int64_t n, double* lab_dev,
                          void* stream);

/* --------------------------------------------------------------- searches */

/* Every passing candidate of one target colour rgb[3] (host), sorted by
 * (k, m), written to out_host[0 .. min(n, cap)) (host).  *n_out receives the
 * number of passing candidates; if it exceeds cap, the first cap records are
 * written and CVS_ERR_TRUNCATED is returned.  target is copied into each
 * record.  Synchronous.  This is the paper's problem statement (§2 Methods):
 * generate the array of pairs, extract those meeting the conditions. */
cvs_status cvs_search_color(cvs_ctx* ctx, const uint8_t rgb[3], uint32_t target,
                            const cvs_grid* grid, const cvs_thresholds* thr,
                            cvs_precision prec, cvs_pair* out_host, size_t cap,
                            size_t* n_out);

/* Every passing pair of n colours (the extraction of cvs_search_color for many
 * targets; for an image, the colours of its pixels, each result being a pure
 * function of the colour): "generate the array, extract the elements that
 * satisfy the conditions" of §1 Introduction and §2 Methods, in one search
 * per batch of colours; each passing pair is written once, straight to its
 * place in the output.
 * rgb_dev: device, 3n bytes.  out_dev: device array of cap records, 16-byte
 * aligned; the pairs of colour i occupy [offsets[i], offsets[i+1]) in (k, m)
 * order, each record's target field = i.  offsets_host: optional host array
 * of n + 1 entries.  *n_out receives the total number of pairs; when it
 * exceeds cap, only the records whose position is below cap are written and
 * CVS_ERR_TRUNCATED is returned (offsets_host and *n_out are still filled, so
 * the call can be repeated with a larger buffer).  n <= 2^31.  Synchronous on
 * `stream`. */
cvs_status cvs_search_colors_pairs(cvs_ctx* ctx, const uint8_t* rgb_dev, int64_t n,
                                   const cvs_grid* grid, const cvs_thresholds* thr,
                                   cvs_precision prec, cvs_pair* out_dev, int64_t cap,
                                   int64_t* offsets_host, int64_t* n_out, void* stream);

/* Per-target results for n colours: for each colour the number of passing
 * candidates, the largest passing radius and the set of patterns that some
 * passing pair carries - the search of §2 Methods (pairs at fixed L*, back to
 * 8-bit RGB, the conditions) reduced to the quantities of Table 2 (which of
 * the Table 1 patterns a colour can carry).  rgb_dev: device, 3n bytes (R,G,B
 * per colour).  out_dev: device capacity map of n entries.  Asynchronous on
 * `stream`; the device buffers must stay valid until it completes. */
cvs_status cvs_search_colors(cvs_ctx* ctx, const uint8_t* rgb_dev, int64_t n,
                             const cvs_grid* grid, const cvs_thresholds* thr,
                             cvs_precision prec, const cvs_capacity_map* out_dev,
                             void* stream);

/* As cvs_search_colors with host buffers: rgb_host (3n bytes), max_r_host,
 * count_host, pmask_host (n entries each).  Copies in, searches and copies
 * out through the context's pinned staging buffers.  Synchronous. */
cvs_status cvs_search_colors_host(cvs_ctx* ctx, const uint8_t* rgb_host, int64_t n,
                                  const cvs_grid* grid, const cvs_thresholds* thr,
                                  cvs_precision prec, float* max_r_host,
                                  int32_t* count_host, uint8_t* pmask_host);

/* Per-colour results for n colours under n_thr threshold sets at once: the
 * experiment of §3 Experiments (Table 1 colours x every (V_th, R_novib)
 * combination), computed in one pass that forms each candidate's pair codes
 * once and decides them against every set.
 *   thr:     host array of n_thr sets, 1 <= n_thr <= 16; all sets must share
 *            gamut_mode (CVS_ERR_INVALID_ARG otherwise).
 *   out_dev: device capacity map of n * n_thr entries; entry t * n_thr + s
 *            holds colour t under set s, equal to what cvs_search_colors
 *            returns for that colour with thr[s] alone.
 *   Each set may carry its own luminance limit (max_dl).
 * Asynchronous on `stream`; not captured in CUDA graphs. */
cvs_status cvs_search_colors_multi(cvs_ctx* ctx, const uint8_t* rgb_dev, int64_t n,
                                   const cvs_grid* grid, const cvs_thresholds* thr,
                                   int32_t n_thr, cvs_precision prec,
                                   const cvs_capacity_map* out_dev, void* stream);

/* Per-pixel results for a batch of n images of any sizes, in one persistent
 * launch over a shared work queue: the search of cvs_search_colors for every
 * pixel's colour (the embedding of Fig. 1a needs, per pixel of the shown
 * image, the pairs that the pixel's colour admits; §2 Methods, Fig. 2).
 * batch: host array of n image descriptors (device pixel pointers).  maps:
 * host array of n capacity maps (device pointers, width*height entries each,
 * row-major, dense).  Asynchronous. */
cvs_status cvs_search_images(cvs_ctx* ctx, const cvs_image* batch, int32_t n,
                             const cvs_grid* grid, const cvs_thresholds* thr,
                             cvs_precision prec, const cvs_capacity_map* maps,
                             void* stream);

/* ---------------------------------------------------------------- embedding
 * The embedding step of Fig. 1a: two frames shown in alternation look like
 * the image to a person, while a camera sees the pixels with information
 * switch between two colours.  Per pixel with requested pattern p (1..7, the
 * Table 1 bit word R,G,B), the pair is the first passing candidate of pattern
 * exactly p in (radius value, radius index k, angle index m) order, i.e. the
 * smallest shift in L*a*b*; frame A gets its "plus" colour (a* + r sin j,
 * b* + r cos j), frame B its "minus" colour.  Pixels whose pattern byte is 0
 * or above 7, and pixels without such a pair, get their own colour in both
 * frames.
 *   img:         device image (HWC bytes, row pitch).
 *   pattern_dev: device bytes, pattern of pixel (x, y) at y * pattern_pitch + x.
 *   frame_a_dev, frame_b_dev: device outputs, HWC bytes, row pitch frame_pitch
 *                (distinct buffers; each may alias img only if frame_pitch
 *                equals its pitch - not recommended).
 *   choice_dev:  optional device output (NULL to skip), width * height dense
 *                uint32: k | m << 16, or 0xFFFFFFFF where nothing was embedded.
 * The thresholds' pattern_mask still applies (a masked pattern never embeds),
 * and so does the luminance limit: with max_dl on, the pair is the first one
 * of pattern p whose two colours also meet it.
 * Asynchronous on `stream`.  cvs_get_stats reports the kernel time; its
 * flagged / rechecked counters count the flagged slots that had to be decided
 * exactly and those re-decided in FP64 (x2 on folded grids). */
cvs_status cvs_embed_image(cvs_ctx* ctx, const cvs_image* img, const uint8_t* pattern_dev,
                           int64_t pattern_pitch, const cvs_grid* grid,
                           const cvs_thresholds* thr, cvs_precision prec,
                           uint8_t* frame_a_dev, uint8_t* frame_b_dev, int64_t frame_pitch,
                           uint32_t* choice_dev, void* stream);

/* An embedding table: the pairs of cvs_embed_image for all 2^24 8-bit
 * colours x 7 patterns, from one search of every colour (radii in sorted
 * order, first hit per pattern).  Afterwards the frames of any image are a
 * gather from the table, identical to cvs_embed_image's on the same grid,
 * thresholds and precision.  The table lives on the context's device
 * (2^24 x 7 entries of 16 bytes = 1.88 GB); the build is synchronous. */
typedef struct cvs_etab cvs_etab;

cvs_status cvs_etab_build(cvs_ctx* ctx, const cvs_grid* grid, const cvs_thresholds* thr,
                          cvs_precision prec, cvs_etab** out, void* stream);

/* Frames (and optionally choices) of one image from the table; arguments and
 * layout as cvs_embed_image.  Asynchronous on `stream`. */
cvs_status cvs_etab_embed_image(cvs_etab* table, const cvs_image* img, const uint8_t* pattern_dev,
                                int64_t pattern_pitch, uint8_t* frame_a_dev, uint8_t* frame_b_dev,
                                int64_t frame_pitch, uint32_t* choice_dev, void* stream);

/* Release a table (waits for the device). */
void cvs_etab_destroy(cvs_etab* table);

/* ------------------------------------------------ colour-keyed memoisation
 * A pixel's result is a pure function of its colour (and of the grid and
 * thresholds).  A capacity table holds the per-colour results of all 2^24
 * 8-bit sRGB colours, computed once by the per-colour search; afterwards the
 * maps of any image are a gather from the table, identical to the maps of
 * cvs_search_images.  The table lives on the context's device (2^24 x 9 bytes
 * plus a small image table) and is independent of the context afterwards. */
typedef struct cvs_lut cvs_lut;

/* Search all 2^24 colours on `grid` with `thr` and store the results in a new
 * table *out (owned by the caller, released with cvs_lut_destroy).  Runs in
 * chunks of 2^22 colours on `stream` and returns when the table is complete. */
cvs_status cvs_lut_build(cvs_ctx* ctx, const cvs_grid* grid, const cvs_thresholds* thr,
                         cvs_precision prec, cvs_lut** out, void* stream);

/* Per-pixel maps of a batch of images from the table (same layout and
 * ownership as cvs_search_images).  Asynchronous on `stream`; one table
 * should be used from one stream at a time. */
cvs_status cvs_lut_lookup_images(cvs_lut* lut, const cvs_image* batch, int32_t n,
                                 const cvs_capacity_map* maps, void* stream);

/* Per-colour results of n colours (rgb_dev: device, 3n bytes) from the table.
 * Asynchronous on `stream`. */
cvs_status cvs_lut_lookup_colors(cvs_lut* lut, const uint8_t* rgb_dev, int64_t n,
                                 const cvs_capacity_map* out, void* stream);

/* Release a table (waits for the device). */
void cvs_lut_destroy(cvs_lut* lut);

/* ------------------------------------------------------------ serving loop
 * A request loop with continuous batching (the paper has no serving loop;
 * this serves its per-pixel search to a stream of frames).  Frames are
 * submitted from host memory at any time; a scheduler thread admits them in
 * arrival order as soon as one of max_inflight slots (each a context and a
 * stream) is free and the device arena has room for the frame and its maps,
 * so frames that arrive while others are on the GPU overlap with them.  The
 * maps of a finished frame stay resident in device memory until released.
 * All device memory (arena, slot scratch for frames up to max_pixels, and the
 * capacity table when use_table = 1) is allocated by cvs_server_create, never
 * during serving.  Host waits are bounded by the caller's timeout. */
typedef struct cvs_server cvs_server;

typedef struct {
    int32_t device;
    int32_t max_inflight;        /* concurrent frames on the device, 1..16 */
    int64_t max_pixels;          /* largest frame accepted (width * height) */
    int64_t mem_budget_bytes;    /* device arena for frames and maps (12 bytes per pixel) */
    int32_t use_table;           /* 1: answer from a capacity table built at creation */
    int32_t dedup;               /* per-frame search (use_table = 0): 1 = one search per
                                    distinct colour of the frame (cvs_set_option "dedup");
                                    its tables, about 130 MB per slot, are allocated at
                                    creation too */
} cvs_server_config;

typedef enum {
    CVS_REQ_QUEUED = 0,
    CVS_REQ_RUNNING = 1,
    CVS_REQ_DONE = 2,
    CVS_REQ_FAILED = 3,
    CVS_REQ_UNKNOWN = 4
} cvs_request_state;

typedef struct {
    int64_t submitted, completed, failed, queued, inflight;
    int64_t bytes_in_use, peak_bytes_in_use;   /* arena */
    double p50_ms, p99_ms, mean_ms, max_ms;    /* submit -> maps resident, completed frames */
    double frames_per_s;                       /* completed / (last completion - first submit) */
} cvs_server_stats;

/* Create a server for one grid, threshold set and precision (copied).
 * Synchronous; with use_table it first builds the capacity table. */
cvs_status cvs_server_create(cvs_server** server, const cvs_server_config* cfg,
                             const cvs_grid* grid, const cvs_thresholds* thr, cvs_precision prec);

/* Stop the scheduler, wait for the device and free everything. */
void cvs_server_destroy(cvs_server* server);

/* Queue a frame (rgb_host: host, HWC bytes, row y at rgb_host + y * pitch).
 * The caller keeps the host frame unchanged until the request is done.
 * *ticket identifies the request.  Never blocks on the device. */
cvs_status cvs_server_submit(cvs_server* server, const uint8_t* rgb_host, int32_t width,
                             int32_t height, int64_t pitch_bytes, uint64_t* ticket);

/* Current cvs_request_state of a ticket. */
cvs_status cvs_server_state(cvs_server* server, uint64_t ticket, int32_t* state);

/* Wait up to timeout_ms for a request to finish: CVS_OK when its maps are
 * resident, CVS_ERR_TIMEOUT if it is still queued or running at the
 * deadline, the request's error if it failed. */
cvs_status cvs_server_wait(cvs_server* server, uint64_t ticket, int32_t timeout_ms);

/* Device pointers of a finished request's maps (width * height entries each,
 * row-major), valid until cvs_server_release. */
cvs_status cvs_server_result(cvs_server* server, uint64_t ticket, cvs_capacity_map* maps,
                             int32_t* width, int32_t* height);

/* Copy a finished request's maps to host buffers (width * height entries
 * each).  Synchronous. */
cvs_status cvs_server_copy_result(cvs_server* server, uint64_t ticket, float* max_r_host,
                                  int32_t* count_host, uint8_t* pmask_host);

/* Drop a request: frees its device memory (a queued request is cancelled; a
 * running one must be waited for first, else CVS_ERR_INVALID_ARG). */
cvs_status cvs_server_release(cvs_server* server, uint64_t ticket);

/* Counters and latency percentiles of the requests so far. */
cvs_status cvs_server_get_stats(cvs_server* server, cvs_server_stats* out);

/* Allocate ahead of time what later searches on this context need: the grid
 * tables of `grid` (may be NULL), scratch for up to max_targets colours or
 * pixels per search, and the image table for batches of up to max_images
 * images, so that those searches make no device allocation (a device
 * allocation synchronises the whole device).  Synchronous. */
cvs_status cvs_reserve(cvs_ctx* ctx, const cvs_grid* grid, int64_t max_targets,
                       int32_t max_images);

/* Wait for the context's work on `stream` and report any device error or
 * device-side timeout.  Fills the counters of the last search. */
cvs_status cvs_synchronize(cvs_ctx* ctx, void* stream);

/* Counters of the last completed search on this context. */
cvs_status cvs_get_stats(cvs_ctx* ctx, cvs_stats* out);

/* Precision study: for n colours (rgb_dev: device, 3n bytes) on the grid,
 * compare every FP32 colour conversion (the "plus" colour of each (k, m), in
 * every FP32 chain the search may take for it) with its FP64 value.
 * Synchronous.  Fields of *out:
 *   max_code_err  largest |v32 - v64| in 8-bit code units among values within
 *                 0.05 of a rounding boundary (v = 255 enc(lin) unrounded)
 *   max_lin_err   largest |lin32 - lin64| of the linear RGB
 *   max_lab_err   largest |a*|, |b*| error of the colour the FP32 chain
 *                 stands for (its f-values against the exact a +- i sin j,
 *                 b +- i cos j); L* is exact
 *   n_wrong_codes FP32 codes in [-1, 256] that differ from FP64 before any
 *                 re-decision
 *   n_unflagged_wrong  of those, the codes the search would take without
 *                 re-deciding them (v32 farther than the context's window W
 *                 from a rounding boundary).  0 means every FP32 decision of
 *                 the search on these colours and this grid is exact: the
 *                 re-decision corrects all the others.
 *   n_values      codes examined
 *   window        the context's window W (option "fp32_window") used */
typedef struct {
    double max_code_err;
    double max_lin_err;
    double max_lab_err;
    int64_t n_wrong_codes;
    int64_t n_values;
    int64_t n_unflagged_wrong;
    double window;
} cvs_precision_report;
cvs_status cvs_precision_probe(cvs_ctx* ctx, const uint8_t* rgb_dev, int64_t n,
                               const cvs_grid* grid, cvs_precision_report* out);

/* A launch shape of the search kernel: threads per block, resident blocks
 * per SM (0 = as many as fit) and radii per work item (a work item is one
 * target x kchunk radii x every angle slot, run by one warp). */
typedef struct {
    int32_t block;
    int32_t blocks_per_sm;
    int32_t kchunk;
    int32_t reserved;
    double ms;            /* search-kernel time of the best shape on the tuning sample */
} cvs_launch_shape;

/* Autotuner: time candidate launch shapes of the per-colour search on these
 * n colours (rgb_dev: device, 3n bytes; at most ~3e10 candidates of them are
 * used per timed launch) and remember the fastest for searches on this
 * context with the same grid, precision, gamut mode and size class (n within
 * a power of two).  *best receives it.  Synchronous; uses the context's own
 * stream.  Shapes set by hand with cvs_set_option take precedence. */
cvs_status cvs_autotune(cvs_ctx* ctx, const uint8_t* rgb_dev, int64_t n, const cvs_grid* grid,
                        const cvs_thresholds* thr, cvs_precision prec, cvs_launch_shape* best);

/* Tuning options of a context (host only):
 *   "fp32_window"   W, the half-width in 8-bit code units of the band around
 *                   a rounding boundary inside which an FP32 code is flagged
 *                   for FP64 re-decision; (0, 0.25); default 2e-3.  It must
 *                   exceed the FP32 path's error for results to be exact.
 *   "block"         threads per block of the search kernel: 64 or 128
 *   "blocks_per_sm" resident blocks per SM (0 = as many as fit)
 *   "kchunk"        radii per work item (0 = automatic)
 *   "autotune"      1: the first search of a new kind (grid, precision, gamut
 *                   mode, size class) times candidate shapes before running,
 *                   as cvs_autotune does; that call then blocks.  Default 0.
 *   "graphs"        1: cvs_search_colors / cvs_search_images capture their
 *                   setup + search + finalize sequence into a CUDA graph the
 *                   first time a given input signature (pointers, sizes, grid,
 *                   thresholds, precision, shape) is seen, and replay the graph
 *                   on later calls with the same signature (up to 8 graphs are
 *                   kept per context).  Default 0.
 *   "dedup"         cvs_search_images searching each distinct colour of the
 *                   batch once (a pixel's maps depend only on its colour) and
 *                   gathering the maps per pixel; the maps are identical.  The
 *                   call then synchronises `stream` once (to size the search)
 *                   and is not captured in a CUDA graph; the context keeps
 *                   about 130 MB of tables for it.  0: never; 1: always (the
 *                   tables are allocated when the option is set); 2 (default):
 *                   for batches of at least 2^20 pixels while option "graphs"
 *                   is 0, when the tables and the search of the distinct
 *                   colours fit the context's memory budget (else the batch
 *                   is searched per pixel and the tables are freed);
 *                   cvs_reserve with max_targets >= 2^20 allocates them if
 *                   they fit.
 *   "angle_ranges"  the FP32 search in gamut-reject mode on a folded, evenly
 *                   spaced angle grid can first turn, per target and radius,
 *                   bounds on the pair's linear RGB (a sinusoid in the angle
 *                   plus a bounded rest) into the angle slots where a pair can
 *                   stay in gamut with a channel able to read high, and then
 *                   search only those slots; results are identical.  The
 *                   multi-threshold search uses the ranges of the union of its
 *                   sets.  0: never; 1: always; 2 (default): not for calls of
 *                   fewer than 8192 (target, radius) pairs, else decided per
 *                   grid, thresholds and kind of call (colours, images, the
 *                   all-colour table, several threshold sets) by a probe of
 *                   4096 targets spread over the first call (which
 *                   synchronises `stream` once), where the ranges list under
 *                   0.6 of the slots the plain search would walk.  The context
 *                   keeps up to 256 MiB of scratch for the ranges.
 *   "fp64_fallback" 1: an FP32_RECHECK call on a grid with a radius above 32
 *                   runs in FP64 instead of returning CVS_ERR_INVALID_ARG.
 *                   Default 0.
 *   "list_batch_items"  pair lists (cvs_search_color, cvs_search_colors_pairs)
 *                   search their colours in batches of at most this many work
 *                   items (a work item: one colour x up to 8192 slots; its
 *                   passing-slot bitmap is kept until its records are
 *                   written; at most 256 MiB of bitmaps per batch); [1, 2^26],
 *                   default 2^22.  Results do not depend on it.
 * Read-only values for cvs_get_option: "graph_launches" (graph replays so
 * far), "graphs_cached", "mem_in_use" (bytes of device memory the context
 * holds), "mem_budget" (the cap given to cvs_create, 0 = none).
 * Unknown names or out-of-range values return CVS_ERR_INVALID_ARG. */
cvs_status cvs_set_option(cvs_ctx* ctx, const char* name, double value);
cvs_status cvs_get_option(cvs_ctx* ctx, const char* name, double* value);

/* ------------------------------------------- allocation-free entry point */

/* cvs_search_colors_noalloc: the per-colour search of cvs_search_colors, for
 * callers that cannot allocate device memory.  The paper has no counterpart to
 * this entry point; it exists for callers such as code hosted inside an
 * application whose memory manager owns the whole device heap and refuses
 * outside cudaMalloc calls, or latency-critical loops in which cudaMalloc's
 * implicit device-wide synchronisation would stall other streams.
 *
 * It takes no context and allocates nothing: no cudaMalloc, no cudaFree and
 * no allocating library routine.  All scratch memory (grid tables, threshold
 * keys, work counters, per-colour constants and accumulators) lives in one
 * fixed array of CVS_NOALLOC_SCRATCH_BYTES inside the library, which every
 * GPU that loads the library holds until the process exits.  The caller
 * passes the inputs and outputs, as for cvs_search_colors: rgb_dev (device,
 * 3n bytes), out_dev (device capacity map of n entries).
 *
 * Limits: n <= CVS_NOALLOC_MAX_COLORS colours, n_radii <=
 * CVS_NOALLOC_MAX_RADII, n_angles <= CVS_NOALLOC_MAX_ANGLES; larger sizes
 * return CVS_ERR_INVALID_ARG with a message naming the limit.
 *
 * The first call on a device looks up the array's device address (once per
 * device; a cudaDeviceReset between calls is not supported): make that first
 * call before any stream capture.  Every call uploads the threshold keys and
 * the grid and reads the angle table back to decide the +180 degree folding,
 * which synchronises `stream`; the search itself then runs asynchronously on
 * `stream`.  All calls share the one array and it keeps the last call's
 * contents (what must start at zero is cleared by each call): calls whose
 * device work overlaps - on different streams or from different threads - race
 * on it, so the caller must serialise them.  The device `device` is made
 * current for the call and the caller's current device is restored before
 * returning.  The luminance limit (thr->max_dl) is not available here (it
 * reads a 128 MiB table) and returns CVS_ERR_INVALID_ARG.  Results are
 * identical to cvs_search_colors on a context with its default options
 * (option "fp32_window" 2e-3). */
#define CVS_NOALLOC_SCRATCH_BYTES (512 * 1024)
#define CVS_NOALLOC_MAX_COLORS 4096
#define CVS_NOALLOC_MAX_RADII 1024
#define CVS_NOALLOC_MAX_ANGLES 1024
cvs_status cvs_search_colors_noalloc(int device, const uint8_t* rgb_dev, int64_t n,
                                     const cvs_grid* grid, const cvs_thresholds* thr,
                                     cvs_precision prec, const cvs_capacity_map* out_dev,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CVSEARCH_H */
