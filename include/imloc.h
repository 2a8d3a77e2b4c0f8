/*
 * imloc.h -- C ABI of the GB300 (sm_103a) implementation of the ImLoc
 * localization hot path: 2D-2D -> 2D-3D lifting through stored depth maps and
 * LO-RANSAC PnP (ImLoc, arXiv 2601.04185, Sec. 3.3).
 *
 * Conventions
 *   - Poses are cam_from_world: X_c = R X_w + t, R row-major 3x3.
 *   - Pixel coordinates are continuous; the image covers [0,W]x[0,H] and the
 *     pixel (i,j) is centred at (i+0.5, j+0.5).
 *   - Depth maps hold z-depth (distance along the optical axis) in float32;
 *     a value <= 0 or non-finite marks "no depth".
 *   - "device" pointers are CUDA global-memory pointers on the context's
 *     device; "host" pointers are ordinary CPU memory.  Every buffer passed in
 *     is owned by the caller and must stay valid until the work enqueued on
 *     `stream` has finished.  The library never frees caller memory and never
 *     returns memory the caller must free.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Functions
 *     named *_async only enqueue work; the others return when the results are
 *     in host memory.
 *   - Every function returns an imloc status (0 = IMLOC_OK, < 0 = error).
 *     Nothing throws across this boundary and nothing aborts the process.
 *   - A context owns one device workspace; calls on one context must not
 *     overlap in time (use one context per concurrent stream).
 */
#ifndef IMLOC_H
#define IMLOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define IMLOC_OK                 0
#define IMLOC_PENDING            1   /* serving: result not ready yet                 */
#define IMLOC_ERR_INVALID_ARG   -1   /* a pointer, size or option is out of range     */
#define IMLOC_ERR_OOM           -2   /* the context workspace (or budget) is too small */
#define IMLOC_ERR_REJECTED      -3   /* serving: admission refused (queue/budget)      */
#define IMLOC_ERR_TIMEOUT       -4   /* a bounded device-side wait gave up             */
#define IMLOC_ERR_CUDA          -5   /* a CUDA runtime call failed                     */
#define IMLOC_ERR_NOT_FOUND     -6   /* serving: unknown or already consumed ticket    */
#define IMLOC_ERR_DEGENERATE    -7   /* fewer than 3 correspondences or no hypothesis  */
#define IMLOC_ERR_CAPACITY      -8   /* an output buffer is smaller than needed        */

typedef struct imloc_ctx imloc_ctx;

/* Create a context on CUDA device `device` with a device workspace of
 * `workspace_bytes` (0 = 512 MiB).  All scratch memory of later calls is
 * carved from this workspace; no later call allocates device memory.  The
 * context also holds 32 MiB of pinned host memory for the small tables a call
 * uploads, used by four calls in turn: an asynchronous call returns once its
 * tables are enqueued and waits on the host only for the uploads of the call
 * four calls back, so the host can enqueue the next calls while the device
 * still runs the earlier ones (their device work stays ordered). */
int imloc_create(imloc_ctx** out, int device, size_t workspace_bytes);
void imloc_destroy(imloc_ctx* ctx);
const char* imloc_status_str(int status);
/* Text of the last failing CUDA runtime call on this thread (for IMLOC_ERR_CUDA). */
const char* imloc_last_cuda_error(void);
/* Sticky device-side error word of the context (IMLOC_OK if none), e.g. a
 * bounded wait that timed out inside a kernel.  Synchronises the context's
 * last stream. */
int imloc_device_error(imloc_ctx* ctx);

/* ---- tracing ----------------------------------------------------------
 * While enabled, every kernel launch of later calls on the context is
 * bracketed by CUDA events on its stream; imloc_profile_read waits for them
 * and returns, per kernel name, the launch count and the summed device time. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} imloc_kernel_stat;

int imloc_profile_enable(imloc_ctx* ctx, int on);
/* Writes min(n, max_out) entries to `out` (host) and the number of kernels
 * seen to *n_out; reset != 0 clears the totals afterwards. */
int imloc_profile_read(imloc_ctx* ctx, imloc_kernel_stat* out, int32_t max_out, int32_t* n_out, int reset);
/* Configuration of the FP32 hypothesis-scoring kernel the context's autotuner
 * chose on its first large enough RANSAC wave (variants differ in speed only,
 * not in results; the paper has no counterpart): CTA threads, poses per thread
 * and poses per work item.  Returns IMLOC_ERR_NOT_FOUND (outputs untouched)
 * before the first tuning; host pointers, any of them may be NULL.
 * Calls with enough pose tiles for two per SM (about 39K minimal sets on 152
 * SMs) score on the tensor cores instead (projection as split-bf16 MMAs, same
 * FP32-level scores up to rounding) and do not tune this kernel; see
 * imloc_set_scoring. */
int imloc_score_config(const imloc_ctx* ctx, int32_t* threads, int32_t* poses_per_thread, int32_t* tile_poses);
/* Scoring kernel of the context's later RANSAC calls (the MSAC scoring of
 * Sec. 3.3; both kernels compute the same FP32-level scores, they differ in
 * speed and in rounding): kernel -1 = by call size (the tensor-core kernel
 * when the call has about two 128-pose tiles per SM; the environment
 * variable IMLOC_SCORE_TC=0 or 1 overrides), 0 = the FP32 kernel, 1 = the
 * tensor-core kernel; tc_variant -1 = default (environment IMLOC_TC_VARIANT),
 * else 0, 1, 2 = records on the MMA's M side (128-record blocks against
 * items of 80, 80 and 64 poses; accumulators read in halves, in quarters
 * with the next one in flight, whole; bf16 pieces), 3 = poses on the M side
 * (80-record blocks against 128-pose tiles, bf16 pieces), 4 = as 3 with TF32
 * pieces.  The continuous-batching
 * server always uses the FP32 kernel.  IMLOC_ERR_INVALID_ARG for a null
 * context or values out of range. */
int imloc_set_scoring(imloc_ctx* ctx, int32_t kernel, int32_t tc_variant);

/* ---- cameras and views -------------------------------------------------- */
typedef struct { float fx, fy, cx, cy; int32_t width, height; } imloc_camera;   /* pinhole */
typedef struct { double R[9]; double t[3]; } imloc_pose;                        /* cam_from_world */

/* Depth map formats of a view. */
#define IMLOC_DEPTH_F32  0  /* float32 metres; <= 0 or non-finite = no depth */
#define IMLOC_DEPTH_LOG8 1  /* 8-bit log codes of imloc_depth_encode_log8_async */
#define IMLOC_DEPTH_F32_TILE4 2  /* float32 metres in 4x4 blocks (imloc_depth_tile4_async) */
#define IMLOC_DEPTH_F32_HALO 3   /* float32 metres in overlapping 8x4 blocks (imloc_depth_halo_async) */

/* One database view of the image-based map (ImLoc Sec. 3.1): a depth map
 * with its intrinsics and pose.  `depth` is a device pointer to height x
 * width values of `depth_format` (float32, or one byte per pixel for
 * IMLOC_DEPTH_LOG8), row stride `pitch` elements; for IMLOC_DEPTH_F32_TILE4
 * and IMLOC_DEPTH_F32_HALO the blocked layouts of imloc_depth_tile4_async and
 * imloc_depth_halo_async, `pitch` = their block-row stride. */
typedef struct {
    const void* depth;
    int32_t width, height;
    int64_t pitch;
    imloc_camera cam;
    imloc_pose pose;
    int32_t depth_format;  /* IMLOC_DEPTH_F32, _LOG8, _F32_TILE4 or _F32_HALO */
    int32_t reserved;      /* 0 */
} imloc_view;

/* ---- depth codec (ImLoc Sec. 3.3 "Data Compression": depth clipped to
 * [0.25 m, 128 m] and quantized in log space with 256 levels; Sec. 4.3
 * "Depth Quantization": under 1.4 % relative error) -----------------------
 * Code 0 = no depth; code c in 1..255 stands for 0.25 * 512^((c-1)/254) m.
 * Encoding maps depth <= 0, NaN or infinite to 0, clips the rest to
 * [0.25, 128] m and rounds to the nearest level in log space (ties to the
 * larger level, decided exactly by comparison with the level midpoints);
 * in-range depths come back within 512^(1/508) - 1 = 1.2357 %.  The lift
 * decodes codes inside its depth fetch (IMLOC_DEPTH_LOG8 views): one byte per
 * tap instead of four, and a map store four times smaller.
 * depth / codes / out: device pointers, row strides in elements; the calls
 * are asynchronous on `stream`, allocate nothing and need no context.
 * IMLOC_ERR_INVALID_ARG on null pointers, width or height < 1 or a stride
 * below the width. */
int imloc_depth_encode_log8_async(const float* depth, int32_t width, int32_t height, int64_t pitch,
                                  uint8_t* codes, int64_t code_pitch, void* stream);
/* codes -> float32 metres (0 for code 0), the same values the lift uses. */
int imloc_depth_decode_log8_async(const uint8_t* codes, int32_t width, int32_t height, int64_t code_pitch,
                                  float* out, int64_t out_pitch, void* stream);

/* ---- blocked float32 depth layout (a storage layout of the map store, not
 * a step of the paper) ---------------------------------------------------
 * The lift's bilinear fetch reads a 2x2 pixel footprint.  In a row-major
 * float32 map it spans two rows, i.e. two DRAM atoms of 64 bytes (three when
 * the pair of columns straddles an atom).  Stored in blocks of 4x4 pixels
 * (64 bytes, one atom), the footprint lies in one block for 9 of 16
 * positions: 1.56 atoms on average instead of 2.13.  Block (bx, by) holds
 * pixels x in [4 bx, 4 bx + 4), y in [4 by, 4 by + 4) in row-major order;
 * pixel (x, y) is element (y / 4) * tiled_pitch + (x / 4) * 16 + (y % 4) * 4
 * + x % 4.  tiled_pitch: elements per block row, a multiple of 16 and
 * >= 16 * ceil(width / 4); the buffer holds ceil(height / 4) * tiled_pitch
 * floats; pixels beyond width / height are written as 0 (no depth).  Written
 * once when a view enters the map store; views with depth_format =
 * IMLOC_DEPTH_F32_TILE4 and pitch = tiled_pitch are lifted with the same
 * values as the row-major map.  Device pointers, asynchronous on `stream`,
 * no allocation, no context; IMLOC_ERR_INVALID_ARG on null pointers, sizes
 * below 1, pitch < width or a bad tiled_pitch. */
int imloc_depth_tile4_async(const float* depth, int32_t width, int32_t height, int64_t pitch, float* tiled,
                            int64_t tiled_pitch, void* stream);

/* ---- overlapping-block float32 depth layout (a storage layout of the map
 * store, not a step of the paper) ---------------------------------------
 * A random depth tap costs the lift a whole 128-byte line of DRAM, so the
 * fewest bytes per match come from every 2x2 bilinear footprint lying in one
 * line.  Blocks of 8x4 pixels (128 bytes) placed every 7 columns and every 3
 * rows overlap by one column and one row, so the footprint with top-left
 * pixel (i, j) lies in block (i / 7, j / 3), and a single lookup at pixel
 * (x, y) reads block (x / 7, y / 3): one line per match, for 32 / 21 = 1.52
 * times the storage of the row-major map.  Block (bx, by) holds pixels
 * x in [7 bx, 7 bx + 8), y in [3 by, 3 by + 4) in row-major order: pixel
 * (7 bx + lx, 3 by + ly) is element by * halo_pitch + bx * 32 + ly * 8 + lx;
 * halo_pitch: elements per block row, a multiple of 32 and
 * >= 32 * ((width - 1) / 7 + 1); the buffer holds ((height - 1) / 3 + 1) *
 * halo_pitch floats; pixels beyond width / height are written as 0 (no
 * depth).  Written once when a view enters the map store; views with
 * depth_format = IMLOC_DEPTH_F32_HALO and pitch = halo_pitch are lifted with
 * the same values as the row-major map.  Device pointers, asynchronous on
 * `stream`, no allocation, no context; IMLOC_ERR_INVALID_ARG on null
 * pointers, sizes below 1, pitch < width or a bad halo_pitch. */
int imloc_depth_halo_async(const float* depth, int32_t width, int32_t height, int64_t pitch, float* halo,
                           int64_t halo_pitch, void* stream);

/* ---- dense triangulation of a mapping depth map (ImLoc Sec. 3.3 "Depth
 * Estimation by Dense Matching") ------------------------------------------
 * Mapping time: the depth map of a reference (mapping) image from its dense
 * matches to n_src covisible source images, all poses known.  Pixel
 * p = j * width + i (centre (i + 0.5, j + 0.5)) has one match per source s:
 * u[s * plane_stride + p], v[...] (source pixel position) and conf[...]
 * (matcher confidence); device arrays.  Per pixel: matches with
 * conf >= conf_min are used; each gives the depth hypothesis where the
 * pixel's ray passes closest to the match's ray; a hypothesis's inliers are
 * the used matches whose angular error (between the match's ray and the
 * direction from its camera centre to the hypothesised point) is below
 * angle_deg; the hypothesis with the most inliers wins (ties: lowest source
 * index); its depth is refined to the minimum of the confidence-weighted
 * squared angular errors of its inliers (Gauss-Newton on the angular error
 * vectors, steps halved until the sum decreases, at most refine_iters);
 * the depth is kept if the inliers number more than keep_more_than.
 * depth_out[p] = reference z-depth in metres (0 = none); inliers_out[p]
 * (may be NULL) = inlier count of the winner.  Asynchronous on `stream`;
 * allocates nothing and needs no context.  IMLOC_ERR_INVALID_ARG for null
 * pointers, n_src outside 1..IMLOC_TRIANGULATE_MAX_SOURCES or a plane
 * stride below width * height. */
#define IMLOC_TRIANGULATE_MAX_SOURCES 16
typedef struct {
    float angle_deg;        /* inlier threshold, 2 degrees */
    float conf_min;         /* 0.05 (matches with conf >= conf_min are used) */
    int32_t keep_more_than; /* 3 */
    int32_t refine_iters;   /* 20 */
} imloc_triangulate_opts;

void imloc_triangulate_default_opts(imloc_triangulate_opts* out);
int imloc_triangulate_depth_async(const imloc_camera* ref_cam, const imloc_pose* ref_pose, int32_t width,
                                  int32_t height, const imloc_camera* src_cams, const imloc_pose* src_poses,
                                  int32_t n_src, const float* u, const float* v, const float* conf,
                                  int64_t plane_stride, const imloc_triangulate_opts* opts, float* depth_out,
                                  uint8_t* inliers_out, void* stream);

/* ---- retrieval nearest-neighbour search (ImLoc Sec. 3.1: a global
 * retrieval feature per database image; Sec. 4.4 "Runtime": the nearest-
 * neighbour search of the retrieval features on the GPU) -----------------
 * queries: n_queries x dim, db: n_db x dim, bfloat16 bit patterns, row-major,
 * device memory, 16-byte aligned; the caller L2-normalises the descriptors,
 * so score = dot product = cosine similarity.  Writes, per query, the k best
 * database rows by descending score (ties: lower index first) to out_score /
 * out_index (device, n_queries x k; slots beyond n_db hold -inf / -1).
 * Scores accumulate in FP32 on the tensor cores (bf16 products are exact).
 * Asynchronous on `stream`; scratch from the context's workspace
 * (4 * min(n_queries, 256) * n_db bytes of scores, n_db rounded up to a
 * multiple of 4, plus the selection buffers).  The order is that of the
 * scores' float bit patterns made monotone, so a NaN score (from non-finite
 * descriptors) ranks above +inf with its sign bit clear, below -inf with it
 * set.  IMLOC_ERR_INVALID_ARG unless 1 <= k <= 128, dim is a positive
 * multiple of 8 and the pointers are 16-byte aligned; IMLOC_ERR_OOM if the
 * workspace is too small. */
int imloc_retrieve_topk_async(imloc_ctx* ctx, const uint16_t* queries, int32_t n_queries, const uint16_t* db,
                              int64_t n_db, int32_t dim, int32_t k, float* out_score, int32_t* out_index,
                              void* stream);

/* ---- lifting (ImLoc Sec. 3.3, "Query Time Matching and 2D-3D Lifting") --
 * A match pairs a query pixel (q_u, q_v) with a database position (db_u,
 * db_v) in one view and carries the matcher confidence.  Matches are grouped
 * in segments of one view and one direction:
 *   direction 0: query->database; (db_u, db_v) is subpixel and the depth is
 *                interpolated bilinearly between the four surrounding pixel
 *                centres (all four must hold a depth and lie inside);
 *   direction 1: database->query; the depth is read at the pixel containing
 *                (db_u, db_v).
 * A match is kept iff conf > 0.05 (compared in float32) and its depth is
 * valid.  Kept matches become correspondences
 *   x, y  = query pixel, X,Y,Z = R^T (d K^-1 [db_u, db_v, 1]^T - t),
 *   w     = conf, src = index of the match in the input,
 * written densely in input order (a stable compaction). */
typedef struct {
    int64_t begin;       /* first match of the segment; the segment ends where the next begins (or at n) */
    int32_t view;        /* index into the view array */
    int32_t direction;   /* 0 = query->database (bilinear), 1 = database->query (lookup) */
} imloc_segment;

typedef struct {
    const float *q_u, *q_v, *db_u, *db_v, *conf; /* device, n each (structure of arrays) */
    int64_t n;
    const imloc_segment* segments;               /* host, n_segments, begins ascending, segments[0].begin == 0 */
    int32_t n_segments;
} imloc_matches;

/* Correspondence set, structure of arrays in device memory (caller-owned).
 * `count` (device, may be NULL on input to RANSAC) holds the number of valid
 * entries; `capacity` bounds every array. */
typedef struct {
    float *x, *y, *X, *Y, *Z, *w;
    int32_t* src;
    int32_t* count;
    int64_t capacity;
} imloc_corr;

/* Lift one query's matches.  Requires out->capacity >= m->n.  Writes the
 * valid count to out->count (device).  Async on `stream`. */
int imloc_lift_async(imloc_ctx* ctx, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                     imloc_corr* out, void* stream);

/* Lift many queries in one launch.  The matches of query q are
 * [query_begin[q], query_begin[q+1]) of `m` (host array, n_queries+1 entries,
 * segment boundaries must include every query boundary).  All outputs go to
 * one concatenated set; the correspondences of query q are
 * [d_offsets[q], d_offsets[q+1]) (device array, n_queries+1 entries). */
int imloc_lift_batch_async(imloc_ctx* ctx, int32_t n_queries, const int64_t* query_begin,
                           const imloc_view* views, int32_t n_views, const imloc_matches* m,
                           imloc_corr* out, int64_t* d_offsets, void* stream);

/* Allocation-free lift (the paper has no counterpart; this is a deployment
 * aid).  For callers that cannot allocate device memory -- code running in a
 * memory pool or budget owned by someone else, processes that reserve all
 * device memory for other components up front, or callers that must not
 * create a context (imloc_create allocates its workspace): it lifts one
 * query exactly like imloc_lift_async but needs no context and performs no
 * allocation.  Its scratch (scan state of the compaction, view, segment and
 * tile tables, an error word; 147,968 bytes) is a fixed array inside the
 * library that every GPU loading the library holds until the process exits.
 *   - Uses the calling thread's current CUDA device.  The first call on a
 *     device looks the array's device address up (cudaGetSymbolAddress) and
 *     keeps it for the process: do not call it again on a device after
 *     cudaDeviceReset there.
 *   - Limits: m->n <= 8,388,608 matches, n_views <= 256, n_segments <= 1024;
 *     larger inputs return IMLOC_ERR_INVALID_ARG without doing any work.
 *   - The view and segment tables are copied from host memory that lives
 *     only during the call, so a call on a stream that is being captured
 *     into a CUDA graph is refused with IMLOC_ERR_INVALID_ARG.
 *   - Every call shares the one array: calls that overlap on the GPU (on
 *     different streams, or from several threads without ordering) race and
 *     give wrong results.  Calls on one stream are ordered and safe.
 *   - If the compaction's bounded wait for a predecessor tile gives up (it
 *     does not in a fault-free run), *out->count (when given) receives
 *     IMLOC_ERR_TIMEOUT instead of the count.
 *   - Host buffers (views, segments) may be freed once the call returns. */
int imloc_lift_noalloc_async(const imloc_view* views, int32_t n_views, const imloc_matches* m, imloc_corr* out,
                             void* stream);

/* ---- LO-RANSAC PnP (ImLoc Sec. 3.3, "Pose Estimation") -----------------
 * Rounds of `batch` minimal sets of 3 correspondences drawn from a uniform
 * stride subsample of at most `max_score_corr` correspondences; every P3P
 * pose is scored by the confidence-weighted truncated squared reprojection
 * error  sum_i w_i min(r_i^2, tau^2)  (a point behind the camera counts
 * tau^2); when a round's best pose beats the best so far, Gauss-Newton LO
 * refines it on the subset; the loop stops after `max_iters` minimal sets or
 * once P(missing the best model) < p_miss; the final pose is refined with a
 * Cauchy loss over all inliers of the full set, weighted by confidence.
 * Minimal sample s of query `query_id` uses Philox4x32-10 with key = seed and
 * counter = (s, query_id, attempt, 0). */
typedef struct {
    double tau_px;           /* inlier threshold in pixels (4) */
    int32_t max_score_corr;  /* subsample cap (10000) */
    int32_t batch;           /* minimal sets per round (1024) */
    int32_t max_iters;       /* minimal sets at most (100000) */
    int32_t lo_iters;        /* Gauss-Newton iterations per LO (10); 0 disables LO */
    double p_miss;           /* adaptive stop (1e-4); <= 0 runs all max_iters */
    int32_t final_iters;     /* Cauchy refinement iterations (25); 0 disables */
    int32_t p3p_fp64_polish; /* 1 (default): Newton polish of the P3P depths with residuals in extended
                                precision (double-float, ~48-bit significand, evaluated on the FP32
                                pipe); 0: FP32 polish */
    double cauchy_scale;     /* Cauchy scale c in pixels (<= 0: use tau_px) */
    uint64_t seed;
    uint32_t query_id;
    int32_t enumerate_all;   /* test mode: every triple of the subset in one round */
    int32_t lo_fp64_accumulate; /* 1: LO / refinement sums each point's normal-equation terms in FP64
                                   (default 0: FP32 per thread, FP64 across warps and CTAs) */
    int32_t lo_fp64_solve;   /* 1: LO / refinement solve their 6x6 normal equations (Cholesky of the
                                Jacobi-scaled system) in FP64 from the FP64 sums; default 0: the same
                                solve in FP32.  The pose itself is kept and updated in FP64 either way */
    int32_t score_bf16;      /* 1: score the minimal-sample poses with bf16-packed subset coordinates
                                (centred and scaled per query) and rescore in FP32 every pair that the
                                bf16 bound cannot classify as an outlier; same scores and counts as the
                                FP32 scoring up to FP32 rounding.  Default 0 */
    int32_t reserved;        /* 0 */
} imloc_ransac_opts;

/* Fill `o` with the defaults above. */
void imloc_ransac_default_opts(imloc_ransac_opts* o);

/* Result of one query (host or device memory, same layout). */
typedef struct {
    double R[9], t[3];           /* final pose (after the Cauchy refinement) */
    double R_best[9], t_best[3]; /* best RANSAC model (after LO), before the refinement */
    double score;                /* its truncated cost on the subset */
    int64_t num_inliers;         /* inliers of the final pose over all correspondences */
    int64_t subset_inliers;      /* inliers of the RANSAC best on the subset */
    int64_t iterations;          /* minimal sets drawn */
    int64_t rounds;
    int64_t lo_count;            /* LO runs */
    int64_t hypotheses;          /* P3P poses scored */
    int64_t best_hyp;            /* 4 * sample + solution index of the last accepted round best */
    int32_t status;              /* IMLOC_OK or IMLOC_ERR_DEGENERATE / IMLOC_ERR_TIMEOUT */
    int32_t passes;              /* diagnostic: reduction passes over the correspondences in LO + refinement */
} imloc_result;

/* One query.  `corr->count` (device) gives N when non-NULL, else
 * corr->capacity is N.  `d_inlier_mask` (device, optional) receives one byte
 * per correspondence: 1 iff inlier of the final pose.  Returns after the
 * result is in `out` (host). */
int imloc_ransac_pnp(imloc_ctx* ctx, const imloc_corr* corr, const imloc_camera* qcam,
                     const imloc_ransac_opts* opts, imloc_result* out, uint8_t* d_inlier_mask, void* stream);

/* Many queries in shared launches.  Query q uses the correspondences
 * [d_offsets[q], d_offsets[q+1]) of the concatenated set `corr` (d_offsets:
 * device, n_queries+1), camera qcams[q] and options opts[q] (host arrays).
 * Results go to d_results[q] (device); masks, if d_masks != NULL, to the
 * device byte array d_masks at the same offsets as the correspondences. */
int imloc_ransac_pnp_batch_async(imloc_ctx* ctx, int32_t n_queries, const imloc_corr* corr,
                                 const int64_t* d_offsets, const imloc_camera* qcams,
                                 const imloc_ransac_opts* opts, imloc_result* d_results,
                                 uint8_t* d_masks, void* stream);

/* ---- generalized absolute pose of a multi-camera rig (ImLoc supplementary
 * "LaMAR HoloLens Results": queries taken by a camera rig) ----------------
 * The query is a rig of n_cams pinhole cameras with known cam_from_rig poses
 * (X_c = R X_r + t); every correspondence carries the index of the camera
 * that observed it (d_cam, device int32, same offsets as the
 * correspondences).  The pose estimated is rig_from_world (X_r = R X_w + t).
 * The loop is that of imloc_ransac_pnp with two changes: the minimal solver
 * is a generalized P3P (the rig poses putting three points on their cameras'
 * rays at positive depth, at most 8 per minimal set, ordered by ascending
 * depth along the first ray; pose id = 8 * sample + solution index), and
 * each residual is the reprojection error in the correspondence's own
 * camera.  Options as imloc_ransac_opts; enumerate_all must be 0,
 * max_iters <= 2^28; p3p_fp64_polish and lo_fp64_accumulate are ignored.
 * Query q uses [d_offsets[q], d_offsets[q+1]) of `corr` and rigs[q] /
 * opts[q] (host arrays).  Results (R, t, R_best, t_best are rig_from_world)
 * go to d_results[q] (device); masks, if d_masks != NULL, as in
 * imloc_ransac_pnp_batch_async.  A query with a camera index outside
 * [0, n_cams) gets status IMLOC_ERR_INVALID_ARG.  Synchronous: returns once
 * the results are written (it reads back one word per wave of rounds). */
#define IMLOC_RIG_MAX_CAMERAS 8
typedef struct {
    int32_t n_cams;                                  /* 1..IMLOC_RIG_MAX_CAMERAS */
    int32_t reserved;
    imloc_camera cams[IMLOC_RIG_MAX_CAMERAS];        /* intrinsics (width/height unused) */
    imloc_pose cam_from_rig[IMLOC_RIG_MAX_CAMERAS];  /* X_c = R X_r + t */
} imloc_rig;

int imloc_ransac_rig_batch(imloc_ctx* ctx, int32_t n_queries, const imloc_corr* corr, const int32_t* d_cam,
                           const int64_t* d_offsets, const imloc_rig* rigs, const imloc_ransac_opts* opts,
                           imloc_result* d_results, uint8_t* d_masks, void* stream);

/* ---- serving: continuous batching (lift + LO-RANSAC PnP) ---------------
 * A server owns a scheduler thread, a device memory pool and a pinned host
 * ring.  Queries are submitted with their matches in HOST memory (copied into
 * the ring before imloc_serve_submit returns) and views whose depth maps are
 * DEVICE memory of a resident map store (they must stay valid until the
 * query's result has been polled).  The scheduler admits queued queries in
 * arrival order while a slot is free and the device pool can hold the
 * query's footprint (matches, correspondences, scratch), lifts them, and
 * advances every resident query by its next RANSAC rounds in shared launches;
 * a query submitted while others run joins at the next step.  Each result
 * equals the one of a plain single-query call up to floating-point
 * reduction order (same Philox samples, same rounds). */
typedef struct imloc_server imloc_server;

typedef struct {
    int32_t max_slots;          /* queries resident on the GPU at once (64) */
    int32_t max_queue;          /* queued, not yet admitted (4096); more: IMLOC_ERR_REJECTED */
    size_t device_budget_bytes; /* device pool for resident queries (1 GiB) */
    size_t host_staging_bytes;  /* pinned ring for submitted matches (256 MiB) */
    int32_t rounds_per_step;    /* RANSAC rounds a resident query advances per step (2; the first step: 1) */
    int32_t reserved;
} imloc_serve_config;

typedef struct {
    int64_t submitted, rejected, admitted, completed, steps, pending, resident;
    size_t device_bytes_in_use;
} imloc_serve_stats;

void imloc_serve_default_config(imloc_serve_config* cfg);
/* Create a server on ctx's device (the server allocates its own pool, ring and
 * internal context; ctx stays free for other calls). */
int imloc_serve_create(imloc_ctx* ctx, const imloc_serve_config* cfg, imloc_server** out);
/* Queue one query.  m: HOST arrays (n matches) and host segments; views: host
 * array of views with device depth maps.  IMLOC_ERR_REJECTED when the queue
 * is full, the staging ring has no room or the query can never fit the
 * device budget. */
int imloc_serve_submit(imloc_server* srv, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                       const imloc_camera* qcam, const imloc_ransac_opts* opts, uint64_t* ticket);
/* The same with the matches already in device memory (m: DEVICE arrays on the
 * server's device, host segments), as a GPU matcher produces them: nothing is
 * copied at submission and the lift reads the arrays in place.  The caller
 * keeps them valid and unchanged until the ticket's result has been polled
 * (or the server is destroyed). */
int imloc_serve_submit_device(imloc_server* srv, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                              const imloc_camera* qcam, const imloc_ransac_opts* opts, uint64_t* ticket);
/* IMLOC_PENDING until done; then IMLOC_OK once with the result (out->status
 * holds the query's own status) and the submit-to-ready latency in ms
 * (optional); IMLOC_ERR_NOT_FOUND for an unknown or already consumed ticket. */
int imloc_serve_poll(imloc_server* srv, uint64_t ticket, imloc_result* out, double* latency_ms);
int imloc_serve_read_stats(imloc_server* srv, imloc_serve_stats* out);
/* Stops the scheduler after its current step; queued and resident queries are dropped. */
int imloc_serve_destroy(imloc_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* IMLOC_H */
