// ctx.h -- host-side context of libimloc: device workspace (bump allocated per
// call), pinned staging buffer for small descriptor uploads, error word.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/imloc.h"

struct imloc_ctx {
    int device = 0;
    int sm_count = 0;
    char* ws = nullptr;           // device workspace
    size_t ws_bytes = 0;
    size_t ws_top = 0;            // bump pointer of the current call
    // pinned host memory for descriptor uploads: a ring of kStagingSlots slots, one per call in turn, so
    // that a call waits (host) only for the uploads of the call kStagingSlots calls back, and the host can
    // enqueue the next calls while the device still runs the previous ones
    static constexpr int kStagingSlots = 4;
    char* staging = nullptr;
    size_t staging_slot_bytes = 0;
    size_t staging_top = 0;       // bump pointer of the current call within its slot
    int staging_slot = 0;         // slot of the current call
    uint64_t call_seq = 0;        // calls begun on this context
    cudaEvent_t staging_free[kStagingSlots] = {};  // per slot: recorded after the last upload that read it
    cudaEvent_t call_done = nullptr;     // recorded after the last call's work; the next call's stream waits on it
    int* d_err = nullptr;         // sticky device error word
    cudaStream_t last_stream = nullptr;
    std::mutex mu;                // serialises calls on one context
    // captured launch sequences of the batched RANSAC, one per size bucket
    std::map<std::string, cudaGraphExec_t> graphs;
    // autotuned score-kernel variant (-1: not tuned yet)
    int score_variant = -1;
    // scoring kernel chosen with imloc_set_scoring (-1: by call size / environment; 0 FP32; 1 tensor cores)
    // and the tensor-core variant (-1: by environment, else the default)
    int scoring_kernel = -1;
    int scoring_tc_variant = -1;
    float score_variant_ms = 0.f;
    // co-resident clusters of the replay kernel (FP32 / FP64 accumulation x cluster size 8 down to 1); 0 = not
    // queried
    int replay_occ[2][8] = {};
    // tracing: CUDA events around every kernel launch while enabled
    bool prof_on = false;
    struct ProfRec { const char* name; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    std::map<std::string, std::pair<int64_t, double>> prof_acc;  // name -> (launches, ms)
};

namespace imloc {

// Start a call on `stream`: reset the bump allocators, take the next staging
// slot and wait (host) until the uploads of its previous use have read it, and
// make `stream` wait for the previous call's device work, which used the same
// workspace.
int begin_call(imloc_ctx* ctx, cudaStream_t stream);
// End a call: record the completion event on `stream`.
int end_call(imloc_ctx* ctx, cudaStream_t stream);
// Device workspace sub-allocation (256-byte aligned); nullptr when it does not fit.
void* ws_alloc(imloc_ctx* ctx, size_t bytes);
// Pinned staging sub-allocation in the call's slot (256-byte aligned); nullptr when it does not fit.
void* staging_alloc(imloc_ctx* ctx, size_t bytes);
// Copy a staged block to the device on `stream`; records the slot's staging event.
int upload(imloc_ctx* ctx, void* d_dst, const void* h_staged, size_t bytes, cudaStream_t stream);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Tracing around one launch: prof_begin records a start event on `stream`
// (no-op when tracing is off); prof_end records the end event.
struct ProfScope {
    imloc_ctx* ctx;
    cudaStream_t stream;
    const char* name;
    cudaEvent_t a = nullptr;
    ProfScope(imloc_ctx* c, cudaStream_t s, const char* n);
    void end();
};

}  // namespace imloc
