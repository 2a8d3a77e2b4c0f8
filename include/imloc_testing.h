/*
 * imloc_testing.h -- test hooks of libimloc: the same kernels as
 * imloc_ransac_pnp, with their intermediate results exposed so that each
 * step of ImLoc Sec. 3.3 "Pose Estimation" (minimal samples, P3P poses,
 * per-pose truncated scores and inlier counts, per-round best) can be
 * compared with an independent implementation.  Same conventions as imloc.h.
 */
#ifndef IMLOC_TESTING_H
#define IMLOC_TESTING_H

#include "imloc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Device buffers (caller-owned; any may be NULL) filled by imloc_testing_ransac.
 * H is the number of minimal sets (opts->max_iters, or C(min(N, cap), 3) in
 * enumerate mode, or n_inject); pose id = 4 * sample + solution index. */
typedef struct {
    int32_t* triples;          /* 3 * H: subset indices of each minimal sample, -1 if degenerate */
    float* poses;              /* 4 * H * 12: pose of each id: R (row-major 3x3) then t */
    float* scores;             /* 4 * H: truncated cost on the subset of each valid pose id */
    int32_t* counts;           /* 4 * H: inliers on the subset of each valid pose id */
    uint64_t* round_best;      /* ceil(H / batch): (score bits << 32) | pose id, ~0 if the round had no pose */
    const float* inject_poses; /* n_inject * 12: score these poses (pose id 4 k) instead of sampling */
    int64_t n_inject;
    uint64_t* rescored_pairs;  /* 1 word, added to: with opts->score_bf16, the (pose, record) pairs that the
                                  bf16 test could not classify as outliers and that were rescored in FP32 */
} imloc_debug;

/* One query with the debug buffers above.  The adaptive stop must be off
 * (opts->p_miss <= 0) so that every round is scored in a single wave; N is
 * corr->capacity (corr->count is ignored).  Synchronous. */
int imloc_testing_ransac(imloc_ctx* ctx, const imloc_corr* corr, const imloc_camera* qcam,
                         const imloc_ransac_opts* opts, const imloc_debug* dbg, imloc_result* out,
                         uint8_t* d_inlier_mask, void* stream);

/* One rig query (imloc_ransac_rig_batch) with the debug buffers above, sized
 * for 8 pose ids per minimal set: poses 8 * H * 12, scores and counts 8 * H
 * (pose id = 8 * sample + solution; ids without a solution hold NaN / -1);
 * injected poses take id 8 k.  The adaptive stop must be off (opts->p_miss
 * <= 0): every round is scored in one wave.  N is corr->capacity; d_cam as
 * in imloc_ransac_rig_batch.  Synchronous. */
int imloc_testing_rig(imloc_ctx* ctx, const imloc_corr* corr, const int32_t* d_cam, const imloc_rig* rig,
                      const imloc_ransac_opts* opts, const imloc_debug* dbg, imloc_result* out,
                      uint8_t* d_inlier_mask, void* stream);

/* The lift of imloc_lift_async with its first `skip_tiles` tiles (1..255)
 * never taken, so that their successors' look-back waits can only end by
 * their iteration limit `spin_limit` (>= 1): exercises the bounded wait and
 * its error report.  The kernel ends; the context's error word then reads
 * IMLOC_ERR_TIMEOUT (imloc_device_error) and the output is not meaningful.
 * Needs more than `skip_tiles` tiles of 1,024 matches. */
int imloc_testing_lift_stalled(imloc_ctx* ctx, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                               imloc_corr* out, int32_t skip_tiles, uint32_t spin_limit, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IMLOC_TESTING_H */
