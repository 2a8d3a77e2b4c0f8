/*
 * imloc_oracle.h -- plain FP64 CPU oracle of the ImLoc localization hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded synthetic inputs.
 *
 * What each function follows (ImLoc, arXiv 2601.04185):
 *   orc_lift          Sec. 3.3 "Query Time Matching and 2D-3D Lifting"
 *   orc_subsample     Sec. 3.3 "Pose Estimation" (uniform subsampling, <=10K)
 *   orc_philox*       counter-based generator (Salmon et al., SC'11), used for
 *                     the minimal samples of Sec. 3.3 "Pose Estimation"
 *   orc_sample        Sec. 3.3 "Pose Estimation" (minimal sets of 3)
 *   orc_p3p           Sec. 3.3 "Pose Estimation" (P3P hypotheses)
 *   orc_score         Sec. 3.3 "Pose Estimation" (truncated squared
 *                     reprojection error weighted by confidence = MSAC)
 *   orc_lo            Sec. 3.3 "Pose Estimation" (LO on a new best)
 *   orc_needed_iters  Sec. 3.3 "Pose Estimation" (stop at 100K iterations or
 *                     when P(missing the best model) < 1e-4)
 *   orc_refine        Sec. 3.3 "Pose Estimation" (final refinement, all
 *                     inliers of the full set, Cauchy loss, confidence weights)
 *   orc_ransac_pnp    the whole loop of Sec. 3.3 "Pose Estimation"
 *   orc_depth_*_log8  Sec. 3.3 "Data Compression" and Sec. 4.3 "Depth
 *                     Quantization" (depth clipped to [0.25, 128] m and
 *                     quantized in log space with 256 levels)
 *   orc_gp3p, orc_rig_*  supplementary "LaMAR HoloLens Results" (generalized
 *                     absolute pose of a multi-camera rig: the Sec. 3.3 loop
 *                     with a generalized P3P and per-camera residuals)
 *   orc_retrieve_topk Sec. 3.1 / Sec. 4.4 "Runtime" (nearest-neighbour
 *                     search of global retrieval features: top-K database
 *                     images by descriptor dot product)
 *   orc_triangulate_* Sec. 3.3 "Depth Estimation by Dense Matching" (per
 *                     pixel: one depth hypothesis per match, most inliers at
 *                     2 degrees, confidence-weighted refinement of the
 *                     squared angular errors, kept with more than 3 inliers)
 *
 * Conventions: poses are cam_from_world, X_c = R X_w + t, R row-major.
 * Pixel coordinates are continuous with the image covering [0,W]x[0,H] and
 * pixel (i,j) centred at (i+0.5, j+0.5).
 */
#ifndef IMLOC_ORACLE_H
#define IMLOC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based generator ------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- lift ---------------------------------------------------------------- */
typedef struct {
    const float* depth;    /* height x width, row stride `pitch` floats; <=0 or non-finite = invalid */
    int64_t width, height, pitch;
    double fx, fy, cx, cy; /* database intrinsics (pixels) */
    double R[9], t[3];     /* database pose, cam_from_world */
} orc_view;

/* Matches are grouped in segments; segment s covers [seg_off[s], seg_off[s+1])
 * and belongs to view seg_view[s] with direction seg_dir[s]:
 *   0 = query->database (database coordinates are subpixel: bilinear depth)
 *   1 = database->query (database coordinates index a pixel: direct lookup).
 * Valid matches are written in input order; returns the count.          */
int64_t orc_lift(const orc_view* views, int64_t n_views,
                 const float* q_u, const float* q_v, const float* db_u, const float* db_v,
                 const float* conf, const int64_t* seg_off, const int32_t* seg_view,
                 const int32_t* seg_dir, int64_t n_seg, float conf_min,
                 double* out_x, double* out_y, double* out_X /* 3 per corr */,
                 double* out_w, int64_t* out_src);

/* ---- RANSAC pieces ------------------------------------------------------ */
void orc_subsample(int64_t n, int64_t m, int64_t* idx);

/* Three distinct indices in [0,m) for minimal sample `sample_id`.
 * Returns the attempt used (0..15), or -1 if all 16 attempts collided.  */
int orc_sample(uint64_t seed, uint32_t query_id, uint32_t sample_id, int64_t m, int64_t out[3]);

/* All real P3P solutions with positive depths for unit bearings y[i] and
 * world points X[i]; sorted by ascending depth of the first point.
 * Returns the count (0..4).                                             */
int orc_p3p(const double y[9], const double X[9], double R_out[36], double t_out[12],
            double lambda_out[12]);

typedef struct {
    int64_t n;
    const double *x, *y; /* observed query pixel */
    const double* X;     /* world points, 3 per corr */
    const double* w;     /* confidence weights */
} orc_corr;

typedef struct { double fx, fy, cx, cy; } orc_cam;

double orc_score(const orc_corr* c, const int64_t* idx, int64_t m, const orc_cam* cam,
                 const double R[9], const double t[3], double tau, int64_t* inliers);

typedef struct {
    double tau;            /* reprojection threshold, pixels */
    int64_t max_score_corr;/* subsample cap, 10000 */
    int64_t batch;         /* minimal sets per round, 1024 */
    int64_t max_iters;     /* 100000 */
    double p_miss;         /* 1e-4; <=0 disables the adaptive stop */
    int64_t lo_iters;      /* Gauss-Newton iterations of one LO, 10 */
    int64_t final_iters;   /* Cauchy IRLS iterations, 25 */
    double cauchy_scale;   /* c of the Cauchy loss, pixels */
    uint64_t seed;
    uint32_t query_id;
    int32_t enumerate_all; /* test mode: every C(m,3) triple, one round */
    int32_t lo_enabled;
    int32_t final_enabled;
} orc_opts;

/* LO on the subset: returns the refined pose and its MSAC score. */
double orc_lo(const orc_corr* c, const int64_t* idx, int64_t m, const orc_cam* cam,
              double tau, int64_t iters, double R[9], double t[3]);

/* Final Cauchy refinement over the fixed set `sel` (indices into c).
 * Returns the number of accepted Gauss-Newton steps.                  */
int orc_refine(const orc_corr* c, const int64_t* sel, int64_t n_sel, const orc_cam* cam,
               double cauchy_c, double tau, int64_t iters, double R[9], double t[3]);

/* Iterations needed so that P(missing the best model) < p_miss with inlier
 * ratio eps and minimal sets of 3.                                     */
double orc_needed_iters(double eps, double p_miss);

typedef struct {
    double R[9], t[3];          /* final pose */
    double R_best[9], t_best[3];/* best RANSAC model before the final refinement */
    double score;               /* MSAC score of that model on the subset */
    int64_t num_inliers;        /* inliers of the final pose over all n */
    int64_t subset_inliers;     /* inliers of the RANSAC best on the subset */
    int64_t iterations;         /* minimal sets drawn */
    int64_t rounds;
    int64_t lo_count;
    int64_t hypotheses;         /* P3P poses scored */
    int64_t best_hyp;           /* pose id (4*sample + k) of the last accepted round-best */
    int32_t status;             /* 0 ok, -1 degenerate */
} orc_result;

/* ---- depth codec ---------------------------------------------------------
 * 8-bit log depth.  Code 0 = no depth; code c in 1..255 stands for the depth
 * 0.25 * 512^((c - 1) / 254) m (255 levels log-uniform over [0.25, 128] m).
 * Encoding: depth <= 0, NaN or infinite -> 0; otherwise the depth is clipped
 * to [0.25, 128] m and rounded to the nearest level in log space (ties to
 * the larger level).                                                      */
double orc_depth_decode_log8(uint8_t code);
uint8_t orc_depth_encode_log8(float depth);
void orc_depth_encode_log8_n(const float* depth, int64_t n, uint8_t* codes);
void orc_depth_decode_log8_n(const uint8_t* codes, int64_t n, double* depth);

/* ---- dense triangulation of a mapping depth map ---------------------------
 * Reference camera (the mapping image) and n_src source cameras with known
 * poses.  Pixel p = j * width + i (centre (i + 0.5, j + 0.5)) carries one match
 * per source s: u[s * stride + p], v[...], conf[...] (source pixel position,
 * confidence).  Per pixel, with X(z) = C0 + z * R0^T K0^-1 [x, y, 1]^T (z the
 * reference z-depth):
 *   - matches with conf >= conf_min are used;
 *   - each used match s gives the hypothesis z_s where the reference ray passes
 *     closest to the source ray (hypotheses with z_s <= 0 or parallel rays are
 *     dropped);
 *   - the inliers of a hypothesis are the used matches whose angular error
 *     angle(X(z) - C_s', ray_s') is below angle_deg;
 *   - the hypothesis with the most inliers wins (ties: the lowest source index);
 *   - its depth is refined to the minimum of sum_{inliers} conf * angle^2
 *     reached by descent from the winning hypothesis: Gauss-Newton steps,
 *     each halved until the sum decreases, until a step is below 1e-14 of the
 *     depth (at most refine_iters steps);
 *   - the depth is kept if the inliers number more than keep_more_than.
 * out_depth[p] = refined z (0 if not kept); out_inliers[p] = inlier count of
 * the winning hypothesis (0 if none).                                       */
typedef struct { double fx, fy, cx, cy; double R[9], t[3]; } orc_tri_cam;
typedef struct {
    double angle_deg;       /* 2 */
    double conf_min;        /* 0.05 */
    int64_t keep_more_than; /* 3 */
    int64_t refine_iters;   /* cap of the descent steps (500: to convergence) */
} orc_tri_opts;

/* Angle (radians) between a and b (atan2 of the cross and dot products). */
double orc_angle(const double a[3], const double b[3]);
/* Closest-approach depth of ray 0 (C0 + z d0) to ray 1 (C1 + l d1); returns
 * 0 for (nearly) parallel rays. */
double orc_closest_depth(const double C0[3], const double d0[3], const double C1[3], const double d1[3]);
/* One pixel; returns the inlier count and writes the depth (0 = none). */
int64_t orc_triangulate_pixel(const orc_tri_cam* ref, int64_t width, int64_t px, int64_t py,
                              const orc_tri_cam* src, int64_t n_src, const double* u, const double* v,
                              const double* conf, const orc_tri_opts* o, double* depth);
void orc_triangulate_depth(const orc_tri_cam* ref, int64_t width, int64_t height, const orc_tri_cam* src,
                           int64_t n_src, const float* u, const float* v, const float* conf, int64_t stride,
                           const orc_tri_opts* o, double* out_depth, int64_t* out_inliers);

/* ---- retrieval nearest-neighbour search -----------------------------------
 * queries: Q x D, db: N x D descriptors as bfloat16 bit patterns (row-major);
 * score(q, n) = sum_d q[d] * db[n][d] (the descriptors are L2-normalised by
 * the caller: cosine similarity).  Top-K per query by descending score, ties
 * to the lower database index; out_score / out_index: Q x K (K <= N).      */
double orc_bf16_to_double(uint16_t bits);
void orc_retrieve_topk(const uint16_t* queries, int64_t Q, const uint16_t* db, int64_t N, int64_t D,
                       int64_t K, double* out_score, int64_t* out_index);

/* ---- generalized absolute pose of a camera rig -----------------------------
 * The rig pose is rig_from_world (X_r = R X_w + t); camera k sees
 * X_c = R[k] X_r + t[k] (cam_from_rig) through intrinsics cam[k].  Every
 * correspondence i belongs to camera cam_of[i].                           */
#define ORC_RIG_MAX_CAMS 8
typedef struct {
    int64_t n_cams;
    orc_cam cam[ORC_RIG_MAX_CAMS];
    double R[ORC_RIG_MAX_CAMS][9];
    double t[ORC_RIG_MAX_CAMS][3];
} orc_rig;

/* GP3P: every rig pose with R X_i + t = o_i + lambda_i d_i, lambda_i > 0, for
 * rays with origins o_i and unit directions d_i in the rig frame; sorted by
 * ascending lambda_1.  Returns the count (0..8).                        */
int orc_gp3p(const double o[9], const double d[9], const double X[9], double R_out[72], double t_out[24],
             double lambda_out[24]);
double orc_rig_score(const orc_corr* c, const int32_t* cam_of, const int64_t* idx, int64_t m, const orc_rig* rig,
                     const double R[9], const double t[3], double tau, int64_t* inliers);
double orc_rig_lo(const orc_corr* c, const int32_t* cam_of, const int64_t* idx, int64_t m, const orc_rig* rig,
                  double tau, int64_t iters, double R[9], double t[3]);
int orc_rig_refine(const orc_corr* c, const int32_t* cam_of, const int64_t* sel, int64_t n_sel, const orc_rig* rig,
                   double cauchy_c, double tau, int64_t iters, double R[9], double t[3]);
/* The loop of orc_ransac_pnp with GP3P hypotheses (pose id = 8 * sample + k)
 * and rig residuals; the result pose is rig_from_world.                  */
int orc_rig_ransac(const orc_corr* c, const int32_t* cam_of, const orc_rig* rig, const orc_opts* o,
                   orc_result* res, uint8_t* inlier_mask, int64_t* round_best_id, double* round_best_score,
                   int64_t max_rounds);

/* Optional per-round trace: round_best_id[r], round_best_score[r]. */
int orc_ransac_pnp(const orc_corr* c, const orc_cam* cam, const orc_opts* o,
                   orc_result* res, uint8_t* inlier_mask,
                   int64_t* round_best_id, double* round_best_score, int64_t max_rounds);

#ifdef __cplusplus
}
#endif
#endif
