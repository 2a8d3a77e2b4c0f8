// ctx.h -- host-side context of libimloc: device workspace (bump allocated per
// call), pinned staging buffer for small descriptor uploads, error word.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>

#include "../../include/imloc.h"

struct imloc_ctx {
    int device = 0;
    int sm_count = 0;
    char* ws = nullptr;           // device workspace
    size_t ws_bytes = 0;
    size_t ws_top = 0;            // bump pointer of the current call
    char* staging = nullptr;      // pinned host memory for descriptor uploads
    size_t staging_bytes = 0;
    size_t staging_top = 0;
    cudaEvent_t staging_free = nullptr;  // recorded after the last upload read the staging buffer
    int* d_err = nullptr;         // sticky device error word
    cudaStream_t last_stream = nullptr;
    std::mutex mu;                // serialises calls on one context
};

namespace imloc {

// Start a call: reset the bump allocators, wait until the previous upload
// has consumed the staging buffer.
int begin_call(imloc_ctx* ctx);
// Device workspace sub-allocation (256-byte aligned); nullptr when it does not fit.
void* ws_alloc(imloc_ctx* ctx, size_t bytes);
// Pinned staging sub-allocation (256-byte aligned); nullptr when it does not fit.
void* staging_alloc(imloc_ctx* ctx, size_t bytes);
// Copy a staged block to the device on `stream`; records the staging event.
int upload(imloc_ctx* ctx, void* d_dst, const void* h_staged, size_t bytes, cudaStream_t stream);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace imloc
