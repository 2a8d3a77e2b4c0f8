// api.cu -- context lifetime, status strings, workspace and staging helpers.
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "ctx.h"

namespace imloc {

static thread_local char g_last_cuda_error[256];

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s:%d %s -> %s", file, line, what,
             cudaGetErrorString(e));
}

int begin_call(imloc_ctx* ctx, cudaStream_t stream) {
    ctx->ws_top = 0;
    ctx->staging_top = 0;
    ctx->staging_slot = static_cast<int>(ctx->call_seq++ % imloc_ctx::kStagingSlots);
    IMLOC_CUDA_TRY(cudaEventSynchronize(ctx->staging_free[ctx->staging_slot]));
    IMLOC_CUDA_TRY(cudaStreamWaitEvent(stream, ctx->call_done, 0));
    return IMLOC_OK;
}

int end_call(imloc_ctx* ctx, cudaStream_t stream) {
    IMLOC_CUDA_TRY(cudaEventRecord(ctx->call_done, stream));
    ctx->last_stream = stream;
    return IMLOC_OK;
}

void* ws_alloc(imloc_ctx* ctx, size_t bytes) {
    size_t off = align_up(ctx->ws_top, 256);
    if (off + bytes > ctx->ws_bytes) return nullptr;
    ctx->ws_top = off + bytes;
    return ctx->ws + off;
}

void* staging_alloc(imloc_ctx* ctx, size_t bytes) {
    size_t off = align_up(ctx->staging_top, 256);
    if (off + bytes > ctx->staging_slot_bytes) return nullptr;
    ctx->staging_top = off + bytes;
    return ctx->staging + static_cast<size_t>(ctx->staging_slot) * ctx->staging_slot_bytes + off;
}

int upload(imloc_ctx* ctx, void* d_dst, const void* h_staged, size_t bytes, cudaStream_t stream) {
    if (bytes == 0) return IMLOC_OK;
    IMLOC_CUDA_TRY(cudaMemcpyAsync(d_dst, h_staged, bytes, cudaMemcpyHostToDevice, stream));
    IMLOC_CUDA_TRY(cudaEventRecord(ctx->staging_free[ctx->staging_slot], stream));
    return IMLOC_OK;
}

static cudaEvent_t prof_event(imloc_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(imloc_ctx* c, cudaStream_t s, const char* n) : ctx(c), stream(s), name(n) {
    if (!ctx->prof_on) return;
    a = prof_event(ctx);
    if (a) cudaEventRecord(a, stream);
}

void ProfScope::end() {
    if (!a) return;
    cudaEvent_t b = prof_event(ctx);
    if (!b) return;
    cudaEventRecord(b, stream);
    ctx->prof_pending.push_back({name, a, b});
    a = nullptr;
}

static void prof_drain(imloc_ctx* ctx) {
    for (auto& r : ctx->prof_pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto& acc = ctx->prof_acc[r.name];
        acc.first += 1;
        acc.second += ms;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
}

}  // namespace imloc

extern "C" {

int imloc_profile_enable(imloc_ctx* ctx, int on) {
    if (!ctx) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->prof_on = on != 0;
    return IMLOC_OK;
}

int imloc_profile_read(imloc_ctx* ctx, imloc_kernel_stat* out, int32_t max_out, int32_t* n_out, int reset) {
    if (!ctx || (max_out > 0 && !out) || !n_out) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    imloc::prof_drain(ctx);
    int32_t k = 0;
    for (auto& kv : ctx->prof_acc) {
        if (k < max_out) {
            memset(&out[k], 0, sizeof(out[k]));
            strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
            out[k].launches = kv.second.first;
            out[k].total_ms = kv.second.second;
        }
        ++k;
    }
    *n_out = k;
    if (reset) ctx->prof_acc.clear();
    return IMLOC_OK;
}

int imloc_create(imloc_ctx** out, int device, size_t workspace_bytes) {
    if (!out) return IMLOC_ERR_INVALID_ARG;
    *out = nullptr;
    int n_dev = 0;
    IMLOC_CUDA_TRY(cudaGetDeviceCount(&n_dev));
    if (device < 0 || device >= n_dev) return IMLOC_ERR_INVALID_ARG;
    IMLOC_CUDA_TRY(cudaSetDevice(device));
    imloc_ctx* c = new imloc_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    c->ws_bytes = workspace_bytes ? workspace_bytes : (size_t(512) << 20);
    c->staging_slot_bytes = size_t(8) << 20;
    if (cudaMalloc(&c->ws, c->ws_bytes) != cudaSuccess) {
        delete c;
        return IMLOC_ERR_OOM;
    }
    bool ok = cudaMallocHost(&c->staging, c->staging_slot_bytes * imloc_ctx::kStagingSlots) == cudaSuccess &&
              cudaMalloc(&c->d_err, sizeof(int)) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->call_done, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < imloc_ctx::kStagingSlots; ++k)
        ok = ok && cudaEventCreateWithFlags(&c->staging_free[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        imloc_destroy(c);
        return IMLOC_ERR_OOM;
    }
    cudaMemset(c->d_err, 0, sizeof(int));
    IMLOC_CUDA_TRY(cudaDeviceSynchronize());
    *out = c;
    return IMLOC_OK;
}

void imloc_destroy(imloc_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    for (int k = 0; k < imloc_ctx::kStagingSlots; ++k)
        if (c->staging_free[k]) cudaEventSynchronize(c->staging_free[k]);
    cudaDeviceSynchronize();
    if (c->ws) cudaFree(c->ws);
    if (c->d_err) cudaFree(c->d_err);
    if (c->staging) cudaFreeHost(c->staging);
    for (int k = 0; k < imloc_ctx::kStagingSlots; ++k)
        if (c->staging_free[k]) cudaEventDestroy(c->staging_free[k]);
    if (c->call_done) cudaEventDestroy(c->call_done);
    for (auto& r : c->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->prof_pool) cudaEventDestroy(e);
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    delete c;
}

const char* imloc_status_str(int s) {
    switch (s) {
        case IMLOC_OK: return "ok";
        case IMLOC_PENDING: return "pending";
        case IMLOC_ERR_INVALID_ARG: return "invalid argument";
        case IMLOC_ERR_OOM: return "out of workspace memory";
        case IMLOC_ERR_REJECTED: return "rejected by admission control";
        case IMLOC_ERR_TIMEOUT: return "bounded device wait timed out";
        case IMLOC_ERR_CUDA: return "CUDA runtime error";
        case IMLOC_ERR_NOT_FOUND: return "unknown ticket";
        case IMLOC_ERR_DEGENERATE: return "degenerate input (fewer than 3 correspondences or no hypothesis)";
        case IMLOC_ERR_CAPACITY: return "output capacity too small";
        default: return "unknown status";
    }
}

int imloc_device_error(imloc_ctx* c) {
    if (!c) return IMLOC_ERR_INVALID_ARG;
    IMLOC_CUDA_TRY(cudaSetDevice(c->device));
    IMLOC_CUDA_TRY(cudaStreamSynchronize(c->last_stream));
    int h = 0;
    IMLOC_CUDA_TRY(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return h == 0 ? IMLOC_OK : IMLOC_ERR_TIMEOUT;
}

const char* imloc_last_cuda_error(void) { return imloc::g_last_cuda_error; }

static_assert(sizeof(imloc_ransac_opts) == 80, "imloc_ransac_opts layout of the header");

void imloc_ransac_default_opts(imloc_ransac_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tau_px = 4.0;
    o->max_score_corr = 10000;
    o->batch = 1024;
    o->max_iters = 100000;
    o->lo_iters = 10;
    o->p_miss = 1e-4;
    o->final_iters = 25;
    o->p3p_fp64_polish = 1;
    o->cauchy_scale = 0.0;
    o->seed = 0;
    o->query_id = 0;
    o->enumerate_all = 0;
}

}  // extern "C"
