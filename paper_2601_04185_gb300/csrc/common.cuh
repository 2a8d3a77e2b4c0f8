// common.cuh -- internal helpers of libimloc (sm_103a): PTX wrappers for
// mbarriers and bulk (TMA) copies with bounded waits, the Philox4x32-10
// generator, warp reductions and the device-side descriptors shared by the
// kernels.  Not part of the public ABI.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/imloc.h"

namespace cg = cooperative_groups;

namespace imloc {

// Sticky device error codes written to the context's error word.
enum DevErr : int {
    kDevOk = 0,
    kDevTimeoutMbar = 1,   // an mbarrier wait exceeded its iteration limit
    kDevTimeoutLookback = 2,// the lift scan waited too long on a predecessor tile
};

// Iteration limit of every spin-wait in this library (each probe of
// mbarrier.try_wait may itself suspend briefly): seconds at most.
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- mbarrier + bulk copy ------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: on timeout record the error and return false; the caller
// carries on with whatever is in shared memory so that every barrier of the
// block (and cluster) is still reached and the kernel ends.  A phase that is
// already complete returns after one non-blocking test.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_test_wait(bar, parity)) return true;
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicCAS(err, 0, kDevTimeoutMbar);
    return false;
}
// One-dimensional bulk copy global -> shared memory of this CTA, completing
// on `bar` (transaction bytes).  Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ---------------------------------
struct U4 { uint32_t x, y, z, w; };
__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
// Minimal sample s of a query: three distinct indices in [0, m) or false.
__device__ __forceinline__ bool draw_triple(uint64_t seed, uint32_t query_id, uint32_t s, uint32_t m, int idx[3]) {
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (uint32_t attempt = 0; attempt < 16; ++attempt) {
        U4 r = philox4x32_10(U4{s, query_id, attempt, 0u}, k0, k1);
        idx[0] = static_cast<int>(__umulhi(r.x, m));
        idx[1] = static_cast<int>(__umulhi(r.y, m));
        idx[2] = static_cast<int>(__umulhi(r.z, m));
        if (idx[0] != idx[1] && idx[0] != idx[2] && idx[1] != idx[2]) return true;
    }
    return false;
}

// ---- warp reductions -------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- scoring records: subset correspondences 2k and 2k+1 interleaved -------
// (48 B, TMA friendly): every field is a float pair, so that one packed
// f32x2 instruction evaluates a pose on both records.  The observed pixel is
// stored negated (the residual is an FMA with it).  An odd subset ends with
// a zero-weight record.
struct __align__(16) ScorePair {
    float X[2], Y[2], Z[2], w[2];  // world points, confidences
    float nx[2], ny[2];            // -observed query pixel
};

struct SubsetRecord {
    float X, Y, Z, w, x, y;
};

__device__ __forceinline__ SubsetRecord subset_record(const ScorePair* s, int64_t i) {
    const ScorePair& p = s[i >> 1];
    const int l = static_cast<int>(i & 1);
    SubsetRecord r;
    r.X = p.X[l]; r.Y = p.Y[l]; r.Z = p.Z[l]; r.w = p.w[l];
    r.x = -p.nx[l]; r.y = -p.ny[l];
    return r;
}

// ---- bf16-packed scoring records (option score_bf16) ----------------------
// Subset records 2k and 2k+1: world coordinates centred and scaled per query,
// X' = (X - c) / s with s a power of two (|X'| <= 1), rounded to bf16 and
// packed in pairs (low half = record 2k); the observed pixels negated in FP32.
// Element 0 of the array is the query's header instead of a pair.
struct __align__(16) ScorePairB {
    uint32_t X2, Y2, Z2, pad;  // bf16 pairs of X', Y', Z'
    float nx[2], ny[2];        // -observed query pixel
};
struct __align__(16) ScoreHeadB {
    float c[3], s;   // centre and scale of the query's subset (bounding box of its records)
    float e;         // bound on |X - (c + s X')| per world coordinate (bf16 and FP32 rounding)
    float xmax, ymax;// max |x|, |y| of the observed pixels
    float wsum;      // sum of the subset's weights
};
static_assert(sizeof(ScorePairB) == 32 && sizeof(ScoreHeadB) == 32, "header in the slot of one pair");

// ---- packed FP32 pairs (fma/mul .f32x2: two IEEE FP32 operations per lane) --
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- hypothesis pose slot: rotation (row-major) + translation, float32 ------
struct __align__(16) PoseF {
    float R[9];
    float t[3];
};

// ---- per-query device descriptor (immutable during a call) ----------------
struct QueryDesc {
    // correspondences (concatenated set): query q reads [off, off + N)
    const float *x, *y, *X, *Y, *Z, *w;
    const int64_t* d_off;   // if non-null: off = d_off[q_off], N = d_off[q_off+1] - off
    const int32_t* d_count; // else if non-null: off = 0, N = *d_count
    int64_t n_host;         // else off = 0, N = n_host
    int32_t q_off;
    int32_t score_bf16;     // score with the bf16-packed records (subset_b) and FP32 rescoring
    uint8_t* mask;          // optional output, same offsets as the correspondences
    imloc_result* result;   // device result slot
    // camera and options
    float fx, fy, cx, cy;
    float ifx_hi, ifx_lo;   // 1/fx as a double-float hi + lo (bearings of the P3P polish)
    float ify_hi, ify_lo;   // 1/fy likewise
    float tau2, cauchy2;
    int32_t m_cap, batch, hyps, rounds;
    int32_t lo_iters, final_iters, polish, enumerate_all;
    int32_t lo_fp64, lo_solve64;  // FP64 accumulation / FP64 6x6 solve in LO and the refinement
    double p_miss;
    uint64_t seed;
    uint32_t query_id;
    int32_t n_cap;          // capacity bound of N (mask / fixed-set buffer)
    // workspace
    ScorePair* subset;      // (m_cap + 1) / 2 record pairs
    float4* tc_rec;         // optional, tensor-core scoring: per subset record (padded to a multiple of
                            // 32) one 128-byte operand row of split TF32 pieces, 128-byte swizzled
    float4* tc_e;           // with tc_rec, tc_mode 0 / 1: per record pair {-x0, -x1, -y0, -y1}, {w0, w1, 0, 0};
                            // tc_mode 2: per record {-x / tau, -y / tau, w tau^2, 0}
    ScorePairB* subset_b;   // option score_bf16: header + (m_cap + 1) / 2 bf16-packed record pairs
    PoseF* slots;           // wave_samples * 4
    int32_t* compact;       // wave_samples * 4 pose ids (valid poses of the wave)
    uint64_t* round_best;   // rounds: (score bits << 32) | pose id, min-reduced
    int32_t* round_hyps;    // rounds: P3P poses produced per round
    int32_t* fixidx;        // fixed inlier set of the final refinement: per replay thread, the indices of its
                            // fixed points at its own positions (same offsets as the correspondences)
    int32_t inject;         // 1: poses are given (one per sample) instead of sampled + solved
    int32_t tc_mode;        // tc_rec rows: 0 TF32 pieces, 1 bf16 pieces, 2 bf16 pieces with 1 in K lane 24 (for
                            // the records-on-M scoring kernel; tc_e per record, see above)
    // optional outputs for the parity tests (one wave only)
    float* score_by_id;     // score of every pose id
    int32_t* count_by_id;   // inlier count of every pose id
    int32_t* triples;       // 3 subset indices per sample (-1 if degenerate)
};

// ---- per-query mutable state -------------------------------------------------
struct QueryState {
    int64_t off, n;          // correspondence offset and count
    int32_t m;               // subset size
    int32_t n_hyp;           // valid poses of the current wave
    double R[9], t[3];       // best model so far
    double best_score;
    int32_t have_best;
    int64_t best_hyp;
    int32_t subset_inliers;
    int32_t rounds_done;
    int64_t iters;
    int64_t hypotheses;
    int32_t lo_count;
    int32_t done;
    int32_t finished;        // final refinement done and result written
    int32_t status;
    int32_t passes;          // reduction passes of LO and refinement (diagnostic)
    int32_t pad;
};

}  // namespace imloc

// host-side error check helper
// On failure: record the call, clear the runtime's last-error state (so that a
// later, unrelated call does not report it again) and return IMLOC_ERR_CUDA.
#define IMLOC_CUDA_TRY(expr)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) {                              \
            imloc::record_cuda_error(_e, #expr, __FILE__, __LINE__); \
            cudaGetLastError();                               \
            return IMLOC_ERR_CUDA;                            \
        }                                                     \
    } while (0)

namespace imloc {
void record_cuda_error(cudaError_t e, const char* what, const char* file, int line);
}
