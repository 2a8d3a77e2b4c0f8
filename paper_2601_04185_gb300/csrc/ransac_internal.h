// ransac_internal.h -- pieces of the LO-RANSAC engine shared by the batched
// entry points (ransac.cu) and the continuous-batching server (serve.cu).
#pragma once

#include "common.cuh"
#include "ctx.h"

namespace imloc {

// Per query and step ("wave"): the minimal samples it draws and the rounds
// the replay walks.
struct WaveQ {
    int64_t s_begin;    // first minimal sample of the step for this query
    int32_t n_samples;  // samples of the step for this query
    int32_t r0, r1;     // rounds [r0, r1) that the replay walks for this query
    int32_t pad;
};

// Device buffers of one launch sequence over nq queries.
struct StepBuffers {
    QueryDesc* d_qd;       // [nq]
    QueryState* d_qs;      // [nq]
    const WaveQ* d_wq;     // [nq] this step
    const int64_t* d_prefix;  // [nq + 1] flattened sample offsets of this step
    int32_t* d_nhyp;       // [nq] valid poses of this step (zero before the step)
    int32_t* d_tiles;      // [3 nq + 1]: item prefix, pose tiles, completed items
    uint32_t* d_counter;   // work queue counter
    int32_t* d_nhyp_all;   // zeroed by the setup kernel (may be null)
    int32_t nhyp_all_len;
    const int32_t* d_init; // queries to set up (null: 0 .. n_init-1)
    bool any_fp64 = false;  // some query asks for FP64 accumulation in LO / refinement
    bool fuse = false;      // replay inside the scoring kernel (see run_step)
    bool tc = false;        // every query has tensor-core operand rows (QueryDesc::tc_rec)
    bool bf16 = false;      // every query scores with bf16-packed records (QueryDesc::subset_b)
    unsigned long long* d_rescored = nullptr;  // bf16 scoring: pairs rescored in FP32 (may be null)
};

// One step: set up n_init queries, then sample + P3P, tiles, score, replay.
int run_step(imloc_ctx* ctx, const StepBuffers& b, int nq, int n_init, int64_t total_samples, bool want_counts,
             cudaStream_t stream);

// Lift of one or more queries (lift.cu), using ctx's workspace for its tables.
int lift_impl(imloc_ctx* ctx, int32_t n_queries, const int64_t* query_begin, const imloc_view* views,
              int32_t n_views, const imloc_matches* m, imloc_corr* out, int64_t* d_offsets, cudaStream_t stream);

}  // namespace imloc
