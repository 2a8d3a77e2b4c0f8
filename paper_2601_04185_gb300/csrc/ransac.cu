// ransac.cu -- GPU LO-RANSAC PnP (ImLoc Sec. 3.3, "Pose Estimation").
//
// The round loop of the method (sample a batch of minimal sets, P3P, score
// every pose on the <= 10K subset, LO when a round's best beats the best so
// far, adaptive stop) is reorganised for the GPU without changing its result:
// minimal sample s is a pure function of (seed, query, s) (counter-based
// Philox), and the score of a pose does not depend on earlier rounds, so all
// rounds of a "wave" are sampled, solved and scored in three wide launches;
// a per-query replay kernel then walks the wave's rounds in order, applies
// the round-best / LO / termination logic exactly as the sequential loop
// would, and runs the final Cauchy refinement once the query is done.  With
// the adaptive stop off a query is one wave; with it on, waves of 1, 1, 2, 4,
// ... rounds bound the speculative work to about twice the rounds needed.
//
// Kernels (in launch order per wave):
//   k_setup        per query: N, subset size M, uniform-stride subset gather
//                  into 48-byte record pairs (and, for tensor-core scoring,
//                  swizzled operand rows of split pieces), reset of the
//                  per-round reductions
//   k_sample_p3p   one minimal sample per thread: Philox triple, bearings,
//                  P3P (FP32 + FP64 Newton polish), pose slots, compact list
//   k_tiles        per-query hypothesis-tile prefix for the work queue
//   k_score        persistent, cluster-split: a cluster takes a (query,
//                  hypothesis tile) from the queue; each CTA of the cluster
//                  keeps its share of the subset resident in shared memory
//                  (bulk copies) and scores HT poses per thread in registers
//                  against two records per packed f32x2 instruction; partial
//                  sums are combined across the cluster
//                  through distributed shared memory; per round, the best
//                  (score, pose id) is kept by a 64-bit atomic minimum
//   k_score_tc     (instead of k_score for large unfused calls) the same
//                  scores with the projection as split-piece tcgen05.mma
//                  into TMEM and the rest of the cost in an FP32 epilogue
//   k_replay       per query (one cluster): rounds in order, LO by
//                  Gauss-Newton on SE(3) (cluster-reduced normal equations,
//                  Jacobi-scaled 6x6 Cholesky), termination, final Cauchy
//                  IRLS.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "p3p.cuh"
#include "ransac_internal.h"
#include "tc.cuh"
#include "../../include/imloc_testing.h"

namespace imloc {


// ============================================================================
// k_setup
// ============================================================================
struct SetupParams {
    const QueryDesc* qd;
    QueryState* qs;
    int32_t* n_hyp_all;       // [waves * nq], zeroed here (may be null)
    int32_t n_hyp_len;
    const int32_t* init_list; // if non-null: block b sets up query init_list[b]
};

constexpr int kSetupBlocks = 8;  // CTAs per query: they split the subset gather
constexpr int kTcBlock = 640;    // tensor-core operand rows are padded to a multiple of this (of every block size)
constexpr uint32_t kBf16Eps = 0x0D80u;  // 2^-100 as bf16 (exponent 27, mantissa 0)
constexpr uint32_t kBf16One = 0x3F80u;  // 1.0 as bf16

// FP32 -> nearest bf16 value (as an FP32)
__device__ __forceinline__ float to_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(lo))) |
           (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(hi))) << 16);
}
// v = p0 + p1 + p2 up to 2^-33 |v| (TF32 pieces) or 2^-26 |v| (bf16 pieces);
// each difference is exact in FP32
__device__ __forceinline__ void split3(float v, bool bf, float& p0, float& p1, float& p2) {
    p0 = bf ? to_bf16(v) : to_tf32(v);
    const float r1 = v - p0;
    p1 = bf ? to_bf16(r1) : to_tf32(r1);
    const float r2 = r1 - p1;
    p2 = bf ? to_bf16(r2) : to_tf32(r2);
}
// which piece of the 4-vector each of the six K terms takes: records
// (b0, b1, b0, b2, b1, b0), poses (a0, a0, a1, a0, a1, a2)
__host__ __device__ constexpr int term_piece(bool pose, int t) {
    return pose ? (t == 2 || t == 4 ? 1 : (t == 5 ? 2 : 0)) : (t == 1 || t == 4 ? 1 : (t == 3 ? 2 : 0));
}
// One 128-byte operand row (8 chunks of 16 bytes, unswizzled order) of the
// 4-vector v: term t (t < 6) holds piece term_piece(pose, t) of v.  TF32: chunk t = term
// t (K = 24 of 32); bf16: chunk c = terms 2c, 2c + 1 (K = 24 of 32).  The
// other chunks are zero.
__device__ __forceinline__ void tc_operand_row(const float v[4], bool bf, bool pose, uint4 ch[8]) {
    float pc[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split3(v[j], bf, pc[0][j], pc[1][j], pc[2][j]);
#pragma unroll
    for (int c = 0; c < 8; ++c) ch[c] = make_uint4(0u, 0u, 0u, 0u);
    if (bf) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* lo = pc[term_piece(pose, 2 * c)];
            const float* hi = pc[term_piece(pose, 2 * c + 1)];
            ch[c] = make_uint4(bf16_pair(lo[0], lo[1]), bf16_pair(lo[2], lo[3]), bf16_pair(hi[0], hi[1]),
                               bf16_pair(hi[2], hi[3]));
        }
    } else {
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const float* pt = pc[term_piece(pose, t)];
            ch[t] = make_uint4(__float_as_uint(pt[0]), __float_as_uint(pt[1]), __float_as_uint(pt[2]),
                               __float_as_uint(pt[3]));
        }
    }
}

__global__ void __launch_bounds__(256) k_setup(const __grid_constant__ SetupParams p) {
    const int qi = blockIdx.x / kSetupBlocks, g = blockIdx.x % kSetupBlocks;
    const int q = p.init_list ? p.init_list[qi] : qi;
    const QueryDesc& d = p.qd[q];
    __shared__ int64_t s_off, s_n;
    __shared__ int32_t s_m;
    if (threadIdx.x == 0) {
        int64_t off = 0, n;
        if (d.d_off) {
            off = d.d_off[d.q_off];
            n = d.d_off[d.q_off + 1] - off;
        } else if (d.d_count) {
            n = *d.d_count;
        } else {
            n = d.n_host;
        }
        QueryState st;
        memset(&st, 0, sizeof(st));
        st.status = IMLOC_OK;
        if (n < 0 || off < 0 || off + n > d.n_cap) {
            n = 0;
            off = 0;
            st.status = IMLOC_ERR_CAPACITY;
        }
        const int32_t m = static_cast<int32_t>(n < d.m_cap ? n : d.m_cap);
        st.off = off;
        st.n = n;
        st.m = m;
        st.best_score = INFINITY;
        st.best_hyp = -1;
        if (n < 3 || d.hyps <= 0) {
            st.done = 1;
            if (st.status == IMLOC_OK) st.status = IMLOC_ERR_DEGENERATE;
        }
        if (g == 0) p.qs[q] = st;
        s_off = off;
        s_n = n;
        s_m = m;
    }
    if (p.n_hyp_all)
        for (int i = blockIdx.x * 256 + threadIdx.x; i < p.n_hyp_len; i += gridDim.x * 256) p.n_hyp_all[i] = 0;
    __syncthreads();
    if (g == 0)
        for (int r = threadIdx.x; r < d.rounds; r += 256) {
            d.round_best[r] = ~0ull;
            d.round_hyps[r] = 0;
        }
    const int64_t off = s_off, n = s_n;
    const int32_t m = s_m;
    // record pair k2 = subset records 2 k2 and 2 k2 + 1 (uniform stride, exact in 64-bit)
    const int m2 = (m + 1) >> 1;
    for (int k2 = g * 256 + threadIdx.x; k2 < m2; k2 += kSetupBlocks * 256) {
        float v[12];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int k = 2 * k2 + l;
            if (k < m) {
                const int64_t i = off + (static_cast<int64_t>(k) * n) / m;
                v[0 + l] = __ldg(d.X + i); v[2 + l] = __ldg(d.Y + i); v[4 + l] = __ldg(d.Z + i);
                v[6 + l] = __ldg(d.w + i); v[8 + l] = -__ldg(d.x + i); v[10 + l] = -__ldg(d.y + i);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) v[2 * c + l] = 0.f;
            }
        }
        float4* dst = reinterpret_cast<float4*>(d.subset + k2);
        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        dst[2] = make_float4(v[8], v[9], v[10], v[11]);
    }
    if (!d.tc_rec) return;
    // Operand rows of the tensor-core scoring: record k is the 4-vector
    // (X, Y, Z, 1) split into pieces b0 + b1 + b2 (TF32 or bf16 values); the
    // row holds the 4-wide terms (b0, b1, b0, b2, b1, b0), matched in the pose
    // rows by (a0, a0, a1, a0, a1, a2), so that one K = 24 product sums the
    // six piece products that carry the FP32 value of a . b.  The row is 128
    // bytes in 16-byte chunks; chunk c of row k sits at position c ^ (k mod 8)
    // (128-byte swizzle of 8-row atoms).  Rows past M up to the next multiple
    // of kTcBlock are zero with weight 0 and a NaN pixel: they add +0 to every
    // score and no inlier.
    const int m_pad = (m + kTcBlock - 1) / kTcBlock * kTcBlock;
    for (int k = g * 256 + threadIdx.x; k < m_pad; k += kSetupBlocks * 256) {
        float c[4] = {0.f, 0.f, 0.f, 0.f}, w = 0.f, nx = __int_as_float(0x7fc00000), ny = nx;
        if (k < m) {
            const int64_t i = off + (static_cast<int64_t>(k) * n) / m;
            c[0] = __ldg(d.X + i); c[1] = __ldg(d.Y + i); c[2] = __ldg(d.Z + i); c[3] = 1.f;
            w = __ldg(d.w + i); nx = -__ldg(d.x + i); ny = -__ldg(d.y + i);
        }
        uint4 ch[8];
        tc_operand_row(c, d.tc_mode != 0, false, ch);
        // mode 2: K lane 24 holds 1 (real records), matched by 2^-100 in the u and v pose rows of k_score_tcr
        if (d.tc_mode == 2 && k < m) ch[3].x = kBf16One;
        uint4* row = reinterpret_cast<uint4*>(d.tc_rec) + static_cast<int64_t>(k) * 8;
        const int sw = k & 7;
#pragma unroll
        for (int j = 0; j < 8; ++j) row[j ^ sw] = ch[j];
        if (d.tc_mode == 2) {
            // pixel scaled by 1 / tau and weight by tau^2 (NaN pixel, weight 0 past M)
            const float inv_tau = 1.0f / sqrtf(d.tau2);
            d.tc_e[k] = make_float4(nx * inv_tau, ny * inv_tau, w * d.tau2, 0.f);
        } else {
            float* e = reinterpret_cast<float*>(d.tc_e + static_cast<int64_t>(k >> 1) * 2);
            const int l = k & 1;
            e[l] = nx;
            e[2 + l] = ny;
            e[4 + l] = w;
            e[6 + l] = 0.f;
        }
    }
}

// ============================================================================
// k_sample_p3p
// ============================================================================
struct SampleParams {
    const QueryDesc* qd;
    const QueryState* qs;
    const WaveQ* wq;            // [nq] of this wave
    const int64_t* prefix;      // [nq+1] flattened sample offsets of this wave
    int32_t* n_hyp;             // [nq] valid poses of this wave
    int64_t total;
    int32_t nq;
};

// lexicographic rank -> triple i < j < k of [0, m) (test mode, small m)
__device__ void unrank_triple(int64_t s, int m, int idx[3]) {
    int i = 0;
    for (; i < m - 2; ++i) {
        const int64_t r = static_cast<int64_t>(m - 1 - i) * (m - 2 - i) / 2;
        if (s < r) break;
        s -= r;
    }
    int j = i + 1;
    for (; j < m - 1; ++j) {
        const int64_t r = m - 1 - j;
        if (s < r) break;
        s -= r;
    }
    idx[0] = i;
    idx[1] = j;
    idx[2] = j + 1 + static_cast<int>(s);
}

__global__ void __launch_bounds__(128) k_sample_p3p(const __grid_constant__ SampleParams p) {
    const int64_t g = static_cast<int64_t>(blockIdx.x) * 128 + threadIdx.x;
    const bool in_range = g < p.total;
    int q = 0;
    if (in_range) {
        int lo = 0, hi = p.nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.prefix[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        q = lo;
    }
    const QueryDesc& d = p.qd[q];
    int nsol = 0;
    int64_t s = 0, local = 0;
    PoseF sol[4];
    if (in_range) {
        local = g - p.prefix[q];
        s = p.wq[q].s_begin + local;
        const QueryState& st = p.qs[q];
        if (d.inject) {
            // poses are given: slot `local` already holds pose 4 s
            nsol = (!st.done && st.m >= 1) ? 1 : 0;
        } else if (!st.done && st.m >= 3) {
            int idx[3];
            bool ok;
            if (d.enumerate_all) {
                unrank_triple(s, st.m, idx);
                ok = true;
            } else {
                ok = draw_triple(d.seed, d.query_id, static_cast<uint32_t>(s), static_cast<uint32_t>(st.m), idx);
            }
            if (d.triples) {
                d.triples[3 * local + 0] = ok ? idx[0] : -1;
                d.triples[3 * local + 1] = ok ? idx[1] : -1;
                d.triples[3 * local + 2] = ok ? idx[2] : -1;
            }
            if (ok) {
                float y[3][3], X[3][3];
                dfloat yd[3][3];
                const float ifx = 1.0f / d.fx, ify = 1.0f / d.fy;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const SubsetRecord c = subset_record(d.subset, idx[k]);
                    const float bx = (c.x - d.cx) * ifx, by = (c.y - d.cy) * ify;
                    const float inv = rsqrtf(bx * bx + by * by + 1.0f);
                    y[k][0] = bx * inv; y[k][1] = by * inv; y[k][2] = inv;
                    X[k][0] = c.X; X[k][1] = c.Y; X[k][2] = c.Z;
                    if (d.polish)
                        bearing_df(c.x, c.y, d.cx, d.cy, dfloat{d.ifx_hi, d.ifx_lo}, dfloat{d.ify_hi, d.ify_lo}, yd[k]);
                }
                float l1[4];
                nsol = p3p_solve(y, d.polish ? yd : nullptr, X, sol, l1);
                for (int k = 0; k < nsol; ++k) d.slots[4 * local + k] = sol[k];
            }
        } else if (d.triples) {
            d.triples[3 * local + 0] = -1;
            d.triples[3 * local + 1] = -1;
            d.triples[3 * local + 2] = -1;
        }
    }
    // append valid pose ids to the query's compact list and count poses per
    // round, aggregated over the lanes of the warp that share the query (and
    // round); full-warp shuffles only
    const int lane = threadIdx.x & 31;
    const int key = in_range ? q : -1;
    const long long rkey = in_range ? ((static_cast<long long>(q) << 32) | (s / d.batch)) : -1ll;
    int excl = 0, total = 0, rtotal = 0, leader = -1, rleader = -1;
    for (int l = 0; l < 32; ++l) {
        const int kl = __shfl_sync(0xffffffffu, key, l);
        const long long rl = __shfl_sync(0xffffffffu, rkey, l);
        const int vl = __shfl_sync(0xffffffffu, nsol, l);
        if (kl == key) {
            if (leader < 0) leader = l;
            if (l < lane) excl += vl;
            total += vl;
        }
        if (rl == rkey) {
            if (rleader < 0) rleader = l;
            rtotal += vl;
        }
    }
    int base = 0;
    if (in_range && lane == leader && total > 0) base = atomicAdd(&p.n_hyp[q], total);
    base = __shfl_sync(0xffffffffu, base, leader < 0 ? lane : leader);
    if (in_range) {
        for (int k = 0; k < nsol; ++k) d.compact[base + excl + k] = static_cast<int32_t>(4 * s + k);
        if (lane == rleader && rtotal > 0) atomicAdd(&d.round_hyps[s / d.batch], rtotal);
    }
}

// ============================================================================
// k_tiles: per-query hypothesis tiles -> exclusive prefix, reset work counter
// ============================================================================
struct TilesParams {
    const QueryState* qs;
    const int32_t* n_hyp;
    int32_t* tile_prefix;  // [nq+1] prefix of items = max(tiles, 1)
    int32_t* ntiles;       // [nq] pose tiles
    int32_t* qdone;        // [nq] zeroed
    uint32_t* work_counter;
    int32_t nq;
    int32_t tile_hyps;
};

__global__ void __launch_bounds__(1024) k_tiles(const __grid_constant__ TilesParams p) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) {
        s_carry = 0;
        *p.work_counter = 0u;
    }
    __syncthreads();
    for (int base = 0; base < p.nq; base += 1024) {
        const int q = base + threadIdx.x;
        int v = 0;
        if (q < p.nq) {
            const int t = p.qs[q].done ? 0 : (p.n_hyp[q] + p.tile_hyps - 1) / p.tile_hyps;
            p.ntiles[q] = t;
            p.qdone[q] = 0;
            v = t > 0 ? t : 1;  // every query has at least one item (its replay trigger)
        }
        int incl = v;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane], wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            s_warp[lane] = wi - w;
        }
        __syncthreads();
        const int excl = s_carry + s_warp[warp] + incl - v;
        if (q < p.nq) p.tile_prefix[q] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) p.tile_prefix[p.nq] = s_carry;
}

// ============================================================================
// k_replay: rounds in order, LO, termination, final refinement
// ============================================================================
// threads per CTA of the stand-alone replay kernel: FP32 accumulation fits
// 128 registers (4 warps per scheduler), FP64 accumulation needs more
template <typename ACC>
__host__ __device__ constexpr int replay_threads() { return sizeof(ACC) == 4 ? 512 : 256; }
constexpr int kMaxReplayThreads = 512;
constexpr int kMaxReplayCluster = 8;
constexpr int kReplayClusterChoices = 8;  // cluster sizes the replay tries (8 down to 1)
constexpr int kNV = 29;  // H (21, upper triangle), g (6), cost, count
constexpr int kPassUnroll = 4;   // correspondences whose loads are in flight together per thread
// shared memory of the stand-alone replay kernel (one CTA per SM) that caches
// each thread's own points: its subset records during LO, its fixed inliers
// during the final refinement (6 floats each, per thread and slot)
constexpr int kReplayStageBytes = 192 * 1024;
constexpr int kKeyCache = 64;    // round minima staged in shared memory at a time

enum PassMode { kLO = 0, kCountSub = 1, kFinInit = 2, kFin = 3, kCountFull = 4 };

// The serial part of the replay (normal-equation solve, pose update, pose
// conversions) sits on the critical path of every Gauss-Newton step.  FP64
// instructions are slow on this part and cost the same for one lane as for
// 32, so the FP64 pose arithmetic is spread over the lanes of warp 0 (one
// output entry per lane) and by default the 6x6 solve runs in FP32 on a
// Jacobi-scaled system: only the step direction depends on it, the fixed
// point of the iteration (zero gradient, FP64 sums) does not.  The option
// lo_fp64_solve solves the same system in FP64 from the FP64 sums.
struct ReplaySmem {
    double R[9], t[3];    // current pose
    double Rc[9], tc[3];  // candidate pose
    double cost, cnt;
    double decrease, prev_cost;
    double need;          // iterations needed by the termination rule at the current inlier ratio
    double tot[32];
    double xch[2][32];
    double red[kMaxReplayThreads / 32][32];
    uint64_t rkey[kKeyCache];
    int32_t rhyps[kKeyCache];
    float Hf[21], gf[6];  // normal equations at the current pose (FP32 copy for the solve)
    float totf[27];
    double Hd[27];        // the same in FP64 (H upper triangle, g) for the FP64 solve
    double dl[6];         // step of the last solve
    double step2;         // its squared norm
    float P[12];
    int flag;
    int skip;             // rounds passed over by the last scan
    float* stg;           // per-thread point cache (null: none): field f, slot j at stg[(f * stg_cap + j) * (NT + 1) + tid]
    int stg_cap;          // slots per thread
    int sub_staged;       // the cache holds this thread's subset records (else: fixed points or nothing)
    int32_t fixcnt[kMaxReplayThreads];  // fixed inliers of each thread (final refinement)
    QueryState st;
};

struct ReplayParams {
    const QueryDesc* qd;
    QueryState* qs;
    const WaveQ* wq;
    int* err;
};

// warp 0: pass pose <- (R, t) in float32 (lane l converts entry l)
__device__ __forceinline__ void pass_pose_warp(ReplaySmem& S, const double* R, const double* t) {
    const int l = threadIdx.x & 31;
    if (l < 12) S.P[l] = static_cast<float>(l < 9 ? R[l] : t[l - 9]);
}

__device__ __forceinline__ float acc_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double acc_fma(double a, double b, double c) { return fma(a, b, c); }

template <int MODE, typename ACC, int NT>
__device__ void pass(ReplaySmem& S, const QueryDesc& d, cg::cluster_group& cluster, int rank, int CL, int& slot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) ++S.st.passes;
    constexpr bool kSub = (MODE == kLO || MODE == kCountSub);
    constexpr bool kJac = (MODE == kLO || MODE == kFinInit || MODE == kFin);
    constexpr int U = kPassUnroll;
    ACC acc[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) acc[k] = ACC(0);
    float Rm[9], tv[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rm[k] = S.P[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) tv[k] = S.P[9 + k];
    const float fx = d.fx, fy = d.fy, cx = d.cx, cy = d.cy, tau2 = d.tau2, c2 = d.cauchy2;
    const float ic2 = 1.0f / c2;
    const int64_t n = kSub ? S.st.m : S.st.n;
    const int64_t off = S.st.off;
    const int64_t stride = static_cast<int64_t>(CL) * NT;
    const int64_t i0 = static_cast<int64_t>(rank) * NT + tid;
    // the thread's points, in order: i0 + j stride (j < nj); in the kFin passes
    // only the fixed inliers among them, whose indices the kFinInit pass
    // recorded at the thread's own positions i0 + k stride (k-th inlier)
    int32_t* fixidx = d.fixidx + off;
    const int64_t nj = (MODE == kFin) ? static_cast<int64_t>(S.fixcnt[tid]) : (n > i0 ? (n - i0 + stride - 1) / stride : 0);
    // the thread's point cache in shared memory: the first J points of the
    // subset (cached by the first subset pass of the call) or of the fixed set
    // (cached by kFinInit); the rest come from global memory
    const int64_t J = S.stg_cap;
    constexpr int64_t SP = NT + 1;  // row stride of the cache: rows of one column fall in different banks
    float* stg = S.stg;
    const bool sub_cached = kSub && S.sub_staged;
    int64_t nfix = 0;
    for (int64_t j0 = 0; j0 < nj; j0 += U) {
        float X[U], Y[U], Z[U], w[U], x[U], y[U];
        int64_t idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u;
            // in the kFin passes: an index this thread wrote in kFinInit (a coherent load)
            idx[u] = j >= nj ? -1
                             : (MODE == kFin ? (j < J ? 0 : static_cast<int64_t>(fixidx[i0 + j * stride]))
                                             : i0 + j * stride);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u;
            const int64_t i = idx[u];
            X[u] = Y[u] = Z[u] = w[u] = x[u] = y[u] = 0.f;
            if (i < 0) continue;
            const bool cached = (MODE == kFin || sub_cached) && j < J;
            if (cached) {
                X[u] = stg[(0 * J + j) * SP + tid]; Y[u] = stg[(1 * J + j) * SP + tid];
                Z[u] = stg[(2 * J + j) * SP + tid]; w[u] = stg[(3 * J + j) * SP + tid];
                x[u] = stg[(4 * J + j) * SP + tid]; y[u] = stg[(5 * J + j) * SP + tid];
            } else if (kSub) {
                const SubsetRecord c = subset_record(d.subset, i);
                X[u] = c.X; Y[u] = c.Y; Z[u] = c.Z; w[u] = c.w; x[u] = c.x; y[u] = c.y;
                if (j < J) {
                    stg[(0 * J + j) * SP + tid] = X[u]; stg[(1 * J + j) * SP + tid] = Y[u];
                    stg[(2 * J + j) * SP + tid] = Z[u]; stg[(3 * J + j) * SP + tid] = w[u];
                    stg[(4 * J + j) * SP + tid] = x[u]; stg[(5 * J + j) * SP + tid] = y[u];
                }
            } else {
                X[u] = __ldg(d.X + off + i); Y[u] = __ldg(d.Y + off + i); Z[u] = __ldg(d.Z + off + i);
                w[u] = __ldg(d.w + off + i); x[u] = __ldg(d.x + off + i); y[u] = __ldg(d.y + off + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = idx[u];
            if (i < 0) break;
            const float xc = fmaf(Rm[0], X[u], fmaf(Rm[1], Y[u], fmaf(Rm[2], Z[u], tv[0])));
            const float yc = fmaf(Rm[3], X[u], fmaf(Rm[4], Y[u], fmaf(Rm[5], Z[u], tv[1])));
            const float zc = fmaf(Rm[6], X[u], fmaf(Rm[7], Y[u], fmaf(Rm[8], Z[u], tv[2])));
            const bool front = zc > 0.f;
            float iz = 0.f, ru = 0.f, rv = 0.f, r2 = tau2;
            if (front) {
                iz = rcp_approx(zc);
                ru = fmaf(fx * xc, iz, cx) - x[u];
                rv = fmaf(fy * yc, iz, cy) - y[u];
                r2 = fmaf(ru, ru, rv * rv);
            }
            const bool inl = front && r2 < tau2;
            float wt = 0.f;
            if (MODE == kLO) {
                acc[27] += w[u] * (inl ? r2 : tau2);
                wt = inl ? w[u] : 0.f;
                acc[28] += inl ? 1.f : 0.f;
            } else if (MODE == kCountSub || MODE == kCountFull) {
                acc[28] += inl ? 1.f : 0.f;
                if (MODE == kCountFull && d.mask) d.mask[off + i] = inl ? 1 : 0;
            } else {
                // kFinInit: the inliers at the initial pose form the fixed set; kFin: a fixed point
                const bool in_set = (MODE == kFin) || inl;
                if (MODE == kFinInit && inl) {
                    if (nfix < J) {
                        stg[(0 * J + nfix) * SP + tid] = X[u]; stg[(1 * J + nfix) * SP + tid] = Y[u];
                        stg[(2 * J + nfix) * SP + tid] = Z[u]; stg[(3 * J + nfix) * SP + tid] = w[u];
                        stg[(4 * J + nfix) * SP + tid] = x[u]; stg[(5 * J + nfix) * SP + tid] = y[u];
                    } else {
                        fixidx[i0 + nfix * stride] = static_cast<int32_t>(i);
                    }
                    ++nfix;
                }
                if (in_set) {
                    const float rr = front ? r2 : tau2;
                    acc[27] += w[u] * c2 * log1pf(rr * ic2);
                    acc[28] += 1.f;
                    wt = front ? w[u] * rcp_approx(fmaf(r2, ic2, 1.0f)) : 0.f;
                }
            }
            if (kJac && wt > 0.f) {
                const float dux = fx * iz, duz = -fx * xc * iz * iz;
                const float dvy = fy * iz, dvz = -fy * yc * iz * iz;
                const float Ju[6] = {duz * yc, dux * zc - duz * xc, -dux * yc, dux, 0.f, duz};
                const float Jv[6] = {-dvy * zc + dvz * yc, -dvz * xc, dvy * xc, 0.f, dvy, dvz};
                // H += w (Ju Ju^T + Jv Jv^T), g += w (Ju ru + Jv rv) as FMA chains; Ju[4] and Jv[3] are
                // zero, so their terms are left out (H[3][4] stays 0)
                int k = 0;
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const float wa = wt * Ju[a], wb = wt * Jv[a];
#pragma unroll
                    for (int b = a; b < 6; ++b) {
                        ACC t = acc[k];
                        if (a != 3 && b != 3) t = acc_fma(ACC(wb), ACC(Jv[b]), t);
                        if (a != 4 && b != 4) t = acc_fma(ACC(wa), ACC(Ju[b]), t);
                        acc[k++] = t;
                    }
                    ACC t = acc[21 + a];
                    if (a != 3) t = acc_fma(ACC(wb), ACC(rv), t);
                    if (a != 4) t = acc_fma(ACC(wa), ACC(ru), t);
                    acc[21 + a] = t;
                }
            }
        }
    }
    if (MODE == kFinInit) S.fixcnt[tid] = static_cast<int32_t>(nfix);
    // block reduction: a transpose butterfly leaves the warp total of value l
    // in lane l (31 shuffles for 32 values), FP64 across warps, then across
    // the CTAs of the cluster in rank order (identical sums in every CTA)
    ACC v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = k < kNV ? acc[k] : ACC(0);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const ACC send = upper ? v[i] : v[i + o];
            const ACC keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    S.red[warp][lane] = static_cast<double>(v[0]);
    __syncthreads();
    if (tid < kNV) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) sum += S.red[w][tid];
        S.xch[slot][tid] = sum;
    }
    cluster.sync();
    if (tid < kNV) {
        double part[kMaxReplayCluster];
#pragma unroll
        for (int r = 0; r < kMaxReplayCluster; ++r)
            part[r] = r < CL ? cluster.map_shared_rank(&S.xch[slot][0], r)[tid] : 0.0;
        double sum = 0.0;
#pragma unroll
        for (int r = 0; r < kMaxReplayCluster; ++r) sum += part[r];
        S.tot[tid] = sum;
        if (tid < 27) S.totf[tid] = static_cast<float>(sum);
    }
    slot ^= 1;
    // every thread read the cache state at the start of the pass (before the first barrier)
    if (tid == 0 && kSub) S.sub_staged = 1;
    if (tid == 0 && MODE == kFinInit) S.sub_staged = 0;
    __syncthreads();
}

__device__ __forceinline__ float solve_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double solve_rsqrt(double v) { return rsqrt(v); }
__device__ __forceinline__ float solve_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double solve_fma(double a, double b, double c) { return fma(a, b, c); }

// (H + mu diag H) x = -g for the 6x6 normal equations (H packed upper
// triangle), after Jacobi scaling D = diag(H)^(-1/2): the scaled matrix has
// the diagonal 1 + mu.  Cholesky of the scaled system in the precision T
// (float: FP32 pipe; double: the FP64 solve of the option lo_fp64_solve);
// returns false if H is not positive definite.
template <typename T>
__device__ __forceinline__ bool solve6(const T* Hu, const T* g, T mu, double x[6], double* dn) {
    T A[6][6], s[6];
    int k = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b) A[a][b] = Hu[k++];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (!(A[a][a] > T(0))) return false;
        s[a] = solve_rsqrt(A[a][a]);
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        A[a][a] = T(1) + mu;
#pragma unroll
        for (int b = a + 1; b < 6; ++b) {
            A[a][b] *= s[a] * s[b];
            A[b][a] = A[a][b];
        }
    }
    T inv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T v = A[i][j];
#pragma unroll
            for (int c = 0; c < j; ++c) v = solve_fma(-A[i][c], A[j][c], v);
            if (i == j) {
                if (!(v > T(0))) return false;
                inv[i] = solve_rsqrt(v);
                A[i][i] = v * inv[i];
            } else {
                A[i][j] = v * inv[j];
            }
        }
    }
    T z[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T v = -g[i] * s[i];
#pragma unroll
        for (int c = 0; c < i; ++c) v = solve_fma(-A[i][c], z[c], v);
        z[i] = v * inv[i];
    }
    T y[6];
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        T v = z[i];
#pragma unroll
        for (int c = i + 1; c < 6; ++c) v = solve_fma(-A[c][i], y[c], v);
        y[i] = v * inv[i];
    }
    T n2 = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const T xi = y[i] * s[i];
        x[i] = static_cast<double>(xi);
        n2 = solve_fma(xi, xi, n2);
    }
    *dn = static_cast<double>(n2);
    return true;
}

// warp 0: candidate (Rc, tc) = Exp(dw) (R, t) + (0, dv) for the step (dw, dv)
// in S.dl, and the pass pose.  Lane l < 9 computes Rc[l], lanes 9..11 tc.
// Exp(dw) = I + A [dw]x + B (dw dw^T - |dw|^2 I), A = sin(th)/th,
// B = (1 - cos(th))/th^2 (Rodrigues), by their Taylor series for th < 0.5
// (remainder < 5e-20) and sincos beyond.
__device__ void apply_step_warp(ReplaySmem& S) {
    const int l = threadIdx.x & 31;
    if (l >= 12) return;
    const double w0 = S.dl[0], w1 = S.dl[1], w2 = S.dl[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B;
    if (th2 < 1e-4) {
        A = 1.0 - th2 * (1.0 / 6.0) * (1.0 - th2 * (1.0 / 20.0) * (1.0 - th2 * (1.0 / 42.0)));
        B = 0.5 - th2 * (1.0 / 24.0) * (1.0 - th2 * (1.0 / 30.0) * (1.0 - th2 * (1.0 / 56.0)));
    } else if (th2 < 0.25) {
        // A = sum_k (-th2)^k / (2k+1)!, B = sum_k (-th2)^k / (2k+2)!, k < 8
        A = 1.0 / 1307674368000.0;  // 1/15!
        B = 1.0 / 20922789888000.0; // 1/16!
        A = 1.0 / 6227020800.0 - th2 * A;  // 1/13!
        B = 1.0 / 87178291200.0 - th2 * B; // 1/14!
        A = 1.0 / 39916800.0 - th2 * A;    // 1/11!
        B = 1.0 / 479001600.0 - th2 * B;   // 1/12!
        A = 1.0 / 362880.0 - th2 * A;      // 1/9!
        B = 1.0 / 3628800.0 - th2 * B;     // 1/10!
        A = 1.0 / 5040.0 - th2 * A;
        B = 1.0 / 40320.0 - th2 * B;
        A = 1.0 / 120.0 - th2 * A;
        B = 1.0 / 720.0 - th2 * B;
        A = 1.0 / 6.0 - th2 * A;
        B = 1.0 / 24.0 - th2 * B;
        A = 1.0 - th2 * A;
        B = 0.5 - th2 * B;
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        A = sn / th;
        B = (1.0 - cs) / th2;
    }
    const int i = l < 9 ? l / 3 : l - 9;
    const double wi = i == 0 ? w0 : (i == 1 ? w1 : w2);
    // row i of [dw]x
    const double k0 = i == 0 ? 0.0 : (i == 1 ? w2 : -w1);
    const double k1 = i == 0 ? -w2 : (i == 1 ? 0.0 : w0);
    const double k2 = i == 0 ? w1 : (i == 1 ? -w0 : 0.0);
    const double c0 = 1.0 - B * th2, bw = B * wi;
    const double e0 = fma(bw, w0, fma(A, k0, i == 0 ? c0 : 0.0));
    const double e1 = fma(bw, w1, fma(A, k1, i == 1 ? c0 : 0.0));
    const double e2 = fma(bw, w2, fma(A, k2, i == 2 ? c0 : 0.0));
    double out;
    if (l < 9) {
        const int j = l - 3 * i;
        out = fma(e0, S.R[j], fma(e1, S.R[3 + j], e2 * S.R[6 + j]));
        S.Rc[l] = out;
    } else {
        out = fma(e0, S.t[0], fma(e1, S.t[1], fma(e2, S.t[2], static_cast<double>(S.dl[3 + i]))));
        S.tc[i] = out;
    }
    S.P[l] = static_cast<float>(out);
}

// warp 0: R <- R (3 I - R^T R) / 2 (Newton-Schulz step towards the nearest
// rotation), lane l < 9 computes entry l; R in shared memory.
__device__ void orthonormalize_warp(double* R) {
    const int l = threadIdx.x & 31;
    const int i = l < 9 ? l / 3 : 0, j = l < 9 ? l - 3 * i : 0;
    // G = R^T R, entry (i, j) in lane 3i + j
    const double g = fma(R[i], R[j], fma(R[3 + i], R[3 + j], R[6 + i] * R[6 + j]));
    const double g0 = __shfl_sync(0xffffffffu, g, j);
    const double g1 = __shfl_sync(0xffffffffu, g, 3 + j);
    const double g2 = __shfl_sync(0xffffffffu, g, 6 + j);
    const double m0 = (j == 0 ? 3.0 : 0.0) - g0, m1 = (j == 1 ? 3.0 : 0.0) - g1, m2 = (j == 2 ? 3.0 : 0.0) - g2;
    const double v = 0.5 * fma(R[3 * i], m0, fma(R[3 * i + 1], m1, R[3 * i + 2] * m2));
    __syncwarp();
    if (l < 9) R[l] = v;
    __syncwarp();
}

__device__ void take_totals(ReplaySmem& S) {
    for (int k = 0; k < 21; ++k) S.Hf[k] = S.totf[k];
    for (int k = 0; k < 6; ++k) S.gf[k] = S.totf[21 + k];
    for (int k = 0; k < 27; ++k) S.Hd[k] = S.tot[k];
    S.cost = S.tot[27];
    S.cnt = S.tot[28];
}

// Gauss-Newton with Marquardt damping retries; starts at S.R, S.t.
template <int INIT, int ITER, typename ACC, int NT>
__device__ void gauss_newton(ReplaySmem& S, const QueryDesc& d, cg::cluster_group& cluster, int rank, int CL, int& slot,
                             int iters) {
    const int tid = threadIdx.x;
    if (tid < 32) pass_pose_warp(S, S.R, S.t);
    __syncthreads();
    pass<INIT, ACC, NT>(S, d, cluster, rank, CL, slot);
    if (tid == 0) take_totals(S);
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        if (S.cnt < 3.0) break;
        bool accepted = false;
        float mu = 0.f;
        for (int attempt = 0; attempt < 4; ++attempt) {
            if (tid == 0)
                S.flag = (d.lo_solve64 ? solve6<double>(S.Hd, S.Hd + 21, static_cast<double>(mu), S.dl, &S.step2)
                                       : solve6<float>(S.Hf, S.gf, mu, S.dl, &S.step2)) ? 1 : 0;
            __syncthreads();
            const bool solved = S.flag != 0;
            if (solved && tid < 32) apply_step_warp(S);
            __syncthreads();
            if (solved) {
                pass<ITER, ACC, NT>(S, d, cluster, rank, CL, slot);
                const bool better = S.tot[27] < S.cost;
                __syncthreads();
                if (better) {
                    if (tid == 0) {
                        S.decrease = S.cost - S.tot[27];
                        S.prev_cost = S.cost;
                        take_totals(S);
                    }
                    if (tid < 12) {
                        if (tid < 9) S.R[tid] = S.Rc[tid];
                        else S.t[tid - 9] = S.tc[tid - 9];
                    }
                    __syncthreads();
                    accepted = true;
                    break;
                }
            }
            mu = (mu == 0.f) ? 1e-3f : mu * 10.f;
        }
        if (!accepted) break;
        // converged: a tiny step, or a step that lowered the cost by < 1e-6 of it
        if (S.step2 < 1e-20 || S.decrease < 1e-6 * S.prev_cost) break;
    }
}

__device__ void write_result(ReplaySmem& S, const QueryDesc& d, int64_t num_inliers) {
    imloc_result r;
    memset(&r, 0, sizeof(r));
    for (int k = 0; k < 9; ++k) { r.R[k] = S.R[k]; r.R_best[k] = S.st.R[k]; }
    for (int k = 0; k < 3; ++k) { r.t[k] = S.t[k]; r.t_best[k] = S.st.t[k]; }
    r.score = S.st.have_best ? S.st.best_score : 0.0;
    r.num_inliers = num_inliers;
    r.subset_inliers = S.st.subset_inliers;
    r.iterations = S.st.iters;
    r.rounds = S.st.rounds_done;
    r.lo_count = S.st.lo_count;
    r.hypotheses = S.st.hypotheses;
    r.best_hyp = S.st.best_hyp;
    r.status = S.st.status;
    r.passes = S.st.passes;
    if (d.result) *d.result = r;
}

// Iterations the termination rule needs at the current subset inlier ratio:
// log(p_miss) / log(1 - eps^3) (INFINITY without a model or for eps = 0).
__device__ double needed_iters(const QueryDesc& d, const QueryState& st) {
    if (!(d.p_miss > 0.0) || !st.have_best || st.m <= 0) return INFINITY;
    const double eps = static_cast<double>(st.subset_inliers) / static_cast<double>(st.m);
    const double e3 = eps * eps * eps;
    if (e3 >= 1.0) return 0.0;
    if (e3 <= 0.0) return INFINITY;
    return log(d.p_miss) / log(1.0 - e3);
}

// Rounds [r0, r1) of one query in order, LO, termination and, once done, the
// final refinement, run by every CTA of one cluster (NT threads each) with
// identical decisions.  Reads and writes the query's state in global memory.
// Rounds whose minimum does not improve on the best score and that do not
// end the search only advance the counters: warp 0 scans the staged round
// minima 32 at a time for the next round that does either.
template <typename ACC, int NT>
__device__ __noinline__ void replay_query(ReplaySmem& S, const QueryDesc& d, QueryState* qs, const WaveQ& wq,
                                          cg::cluster_group& cluster, int CL, int rank) {
    static_assert(sizeof(QueryState) % 8 == 0, "state copied in 8-byte words");
    constexpr int kWords = static_cast<int>(sizeof(QueryState) / 8);
    const int tid = threadIdx.x;
    const int r_end = min(wq.r1, d.rounds);
    int c0 = wq.r0, c1 = min(wq.r0 + kKeyCache, r_end);  // staged rounds [c0, c1)
    __syncthreads();
    if (tid == 0) S.sub_staged = 0;
    for (int k = tid; k < kWords; k += NT)
        reinterpret_cast<uint64_t*>(&S.st)[k] = reinterpret_cast<const uint64_t*>(qs)[k];
    // the round minima (all final: the scoring of the wave is complete)
    for (int k = tid; k < c1 - c0; k += NT) {
        S.rkey[k] = d.round_best[c0 + k];
        S.rhyps[k] = d.round_hyps[c0 + k];
    }
    __syncthreads();
    if (tid == 0) S.need = needed_iters(d, S.st);
    // every CTA holds its copy of the state before rank 0 can write it back
    cluster.sync();
    if (S.st.finished) return;  // same decision in every CTA of the cluster
    int slot = 0;
    int r = wq.r0;
    while (r < r_end && !S.st.done) {
        if (r >= c1) {
            __syncthreads();
            c0 = r;
            c1 = min(r + kKeyCache, r_end);
            for (int k = tid; k < c1 - c0; k += NT) {
                S.rkey[k] = d.round_best[c0 + k];
                S.rhyps[k] = d.round_hyps[c0 + k];
            }
            __syncthreads();
        }
        if (tid < 32) {
            // next event among the staged rounds: an improving minimum or a stop
            int e = c1 - r;
            for (int base = r; base < c1; base += 32) {
                const int rr = base + tid;
                bool ev = false;
                if (rr < c1) {
                    const uint64_t key = S.rkey[rr - c0];
                    const bool imp = key != ~0ull &&
                                     static_cast<double>(__uint_as_float(static_cast<uint32_t>(key >> 32))) <
                                         S.st.best_score;
                    const int64_t it = min(static_cast<int64_t>(rr + 1) * d.batch, static_cast<int64_t>(d.hyps));
                    ev = imp || it >= d.hyps || static_cast<double>(it) >= S.need;
                }
                const unsigned m = __ballot_sync(0xffffffffu, ev);
                if (m != 0u) {
                    e = base + __ffs(m) - 1 - r;
                    break;
                }
            }
            long long hs = 0;
            for (int k = tid; k < e; k += 32) hs += S.rhyps[r - c0 + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, o);
            if (tid == 0) {
                if (e > 0) {
                    S.st.hypotheses += hs;
                    S.st.iters = min(static_cast<int64_t>(r + e) * d.batch, static_cast<int64_t>(d.hyps));
                    S.st.rounds_done = r + e;
                }
                S.skip = e;
            }
        }
        __syncthreads();
        r += S.skip;
        if (r >= c1) continue;
        // round r: its minimum improves on the best score, or the search stops after it
        const uint64_t key = S.rkey[r - c0];
        const int hyps_r = S.rhyps[r - c0];
        bool improve = false;
        float sc = 0.f;
        if (key != ~0ull) {
            sc = __uint_as_float(static_cast<uint32_t>(key >> 32));
            improve = static_cast<double>(sc) < S.st.best_score;
        }
        __syncthreads();  // every thread has read the best score before it changes
        if (improve) {
            if (tid < 32) {
                const int l = tid;
                const uint32_t id = static_cast<uint32_t>(key & 0xffffffffu);
                const PoseF& ps = d.slots[static_cast<int64_t>(id) - 4 * wq.s_begin];
                if (l < 9) S.R[l] = ps.R[l];
                else if (l < 12) S.t[l - 9] = ps.t[l - 9];
                __syncwarp();
                // float32 pose -> rotation to FP64 rounding (quadratic convergence from ~1e-7)
                orthonormalize_warp(S.R);
                orthonormalize_warp(S.R);
                if (l < 9) S.st.R[l] = S.R[l];
                else if (l < 12) S.st.t[l - 9] = S.t[l - 9];
                if (l == 0) {
                    S.st.best_score = sc;
                    S.st.best_hyp = id;
                    S.st.have_best = 1;
                }
            }
            __syncthreads();
            if (d.lo_iters > 0) {
                gauss_newton<kLO, kLO, ACC, NT>(S, d, cluster, rank, CL, slot, d.lo_iters);
                if (tid == 0) {
                    ++S.st.lo_count;
                    if (S.cost < S.st.best_score) {
                        for (int k = 0; k < 9; ++k) S.st.R[k] = S.R[k];
                        for (int k = 0; k < 3; ++k) S.st.t[k] = S.t[k];
                        S.st.best_score = S.cost;
                    }
                    S.st.subset_inliers = static_cast<int32_t>(S.cnt);
                }
            } else {
                if (tid < 32) pass_pose_warp(S, S.st.R, S.st.t);
                __syncthreads();
                pass<kCountSub, float, NT>(S, d, cluster, rank, CL, slot);
                if (tid == 0) S.st.subset_inliers = static_cast<int32_t>(S.tot[28]);
            }
            if (tid == 0) S.need = needed_iters(d, S.st);
            __syncthreads();
        }
        if (tid == 0) {
            const int64_t it = min(static_cast<int64_t>(r + 1) * d.batch, static_cast<int64_t>(d.hyps));
            S.st.iters = it;
            S.st.rounds_done = r + 1;
            S.st.hypotheses += hyps_r;
            if (it >= d.hyps || static_cast<double>(it) >= S.need) S.st.done = 1;
        }
        __syncthreads();
        ++r;
    }
    if (S.st.done && !S.st.finished) {
        if (!S.st.have_best) {
            if (tid == 0) {
                if (S.st.status == IMLOC_OK) S.st.status = IMLOC_ERR_DEGENERATE;
                for (int k = 0; k < 9; ++k) S.R[k] = (k % 4 == 0) ? 1.0 : 0.0;
                for (int k = 0; k < 3; ++k) S.t[k] = 0.0;
                if (rank == 0) write_result(S, d, 0);
                S.st.finished = 1;
            }
            __syncthreads();
        } else {
            if (tid < 12) {
                if (tid < 9) S.R[tid] = S.st.R[tid];
                else S.t[tid - 9] = S.st.t[tid - 9];
            }
            __syncthreads();
            if (d.final_iters > 0) gauss_newton<kFinInit, kFin, ACC, NT>(S, d, cluster, rank, CL, slot, d.final_iters);
            if (tid < 32) pass_pose_warp(S, S.R, S.t);
            __syncthreads();
            pass<kCountFull, float, NT>(S, d, cluster, rank, CL, slot);
            const int64_t num_inliers = static_cast<int64_t>(S.tot[28]);
            if (tid == 0) {
                if (rank == 0) write_result(S, d, num_inliers);
                S.st.finished = 1;
            }
            __syncthreads();
        }
    }
    if (rank == 0)
        for (int k = tid; k < kWords; k += NT)
            reinterpret_cast<uint64_t*>(qs)[k] = reinterpret_cast<const uint64_t*>(&S.st)[k];
    __syncthreads();
}

// Stand-alone replay: one cluster per query (queries whose accumulation
// precision this instance implements; the others are skipped).
template <typename ACC>
__global__ void __launch_bounds__(replay_threads<ACC>()) k_replay(const __grid_constant__ ReplayParams p) {
    __shared__ ReplaySmem S;
    extern __shared__ __align__(16) float replay_stage[];
    constexpr int NT = replay_threads<ACC>();
    if (threadIdx.x == 0) {
        S.stg = replay_stage;
        S.stg_cap = kReplayStageBytes / (6 * static_cast<int>(sizeof(float)) * (NT + 1));
    }
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int q = blockIdx.x / CL;
    const QueryDesc& d = p.qd[q];
    if ((d.lo_fp64 != 0) == (sizeof(ACC) == 8)) replay_query<ACC, replay_threads<ACC>()>(S, d, p.qs + q, p.wq[q], cluster, CL, rank);
    // no CTA may leave while another can still read its shared memory
    cluster.sync();
}

// ============================================================================
// k_score: persistent, cluster-split hypothesis scoring
// ============================================================================
constexpr int kChunkPairs = 128;   // subset record pairs per bulk copy (6 KB)
constexpr int kScoreCluster = 8;   // CTAs per (query, pose tile) item: they split the subset
constexpr int kWinPairs = 640;     // record pairs resident per CTA (30 KB): M <= 10,240 in one window
constexpr int kWinChunks = kWinPairs / kChunkPairs;
constexpr int kMaxTileHyps = 512;  // poses per item: THREADS x HT of the variant, at most this

struct ScoreParams {
    const QueryDesc* qd;
    QueryState* qs;
    const WaveQ* wq;
    const int32_t* n_hyp;
    const int32_t* tile_prefix;  // [nq + 1] items: max(tiles, 1) per query
    const int32_t* ntiles;       // [nq] pose tiles per query (0 for a finished query)
    int32_t* qdone;              // [nq] items completed (fused replay trigger)
    uint32_t* work_counter;
    int32_t nq;
    int* err;
    unsigned long long* rescored;  // bf16 scoring: (pose, record) pairs rescored in FP32 (may be null)
};

// Each CTA keeps its share of the query's subset resident in shared memory:
// one bulk copy (and one mbarrier) per 128-pair chunk, so compute starts on
// chunk 0 while the rest lands, no block barrier between chunks, and the
// next item of the same query reuses the data.  Every thread scores HT poses
// held in registers against every record pair of the share: the projection
// and the residual (13 of the 14 FP32-pipe operations per pose and record)
// run as fma/mul.f32x2 on both records of a pair (the pose coefficients are
// duplicated into both halves; the observed pixels of a pair are stored as
// pairs), the reciprocal, the truncation and the weighted sum in scalar FP32
// on the unpacked halves, so that the issue slots the packed instructions
// free serve the reciprocal, min/max and shared-memory loads.  Per
// chunk, the even and the odd records of the chunk are summed separately, in
// order, and the chunk adds even + odd to the pose's total: the partial sums
// do not depend on (THREADS, HT).
// FUSED: after its last item of a query, a cluster replays that query
// (round-best / LO / termination / refinement) while other clusters keep
// scoring: the replay needs no separate launch and overlaps the scoring.
template <int THREADS, int HT, bool COUNT, int MINB, int UNR, bool FUSED, int MINB_FUSED>
__global__ void __launch_bounds__(THREADS, FUSED ? MINB_FUSED : MINB) k_score(const __grid_constant__ ScoreParams p) {
    constexpr int TH = THREADS * HT;  // poses per item
    static_assert(TH <= kMaxTileHyps && TH % kScoreCluster == 0, "tile size");
    extern __shared__ __align__(128) unsigned char smem[];
    ScorePair* buf = reinterpret_cast<ScorePair*>(smem);
    float* s_part = reinterpret_cast<float*>(buf + kWinPairs);
    int* s_cnt = reinterpret_cast<int*>(s_part + TH);
    __shared__ __align__(8) uint64_t bar[kWinChunks];
    __shared__ int s_item, s_last;
    __shared__ ReplaySmem S_rep;

    cg::cluster_group cluster = cg::this_cluster();
    const int CS = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int c = 0; c < kWinChunks; ++c) mbar_init(&bar[c], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t phases = 0u;           // parity bit per chunk barrier
    int loaded_q = -1, loaded_w0 = -1, loaded_n = -1;
    const int total_tiles = p.tile_prefix[p.nq];

    for (;;) {
        if (rank == 0 && tid == 0) s_item = static_cast<int>(atomicAdd(p.work_counter, 1u));
        cluster.sync();
        const int item = *cluster.map_shared_rank(&s_item, 0);
        cluster.sync();
        if (item >= total_tiles) break;
        int lo = 0, hi = p.nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.tile_prefix[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int q = lo;
        const int tile = item - p.tile_prefix[q];
        const QueryDesc& d = p.qd[q];
        if (tile < p.ntiles[q]) {
        const int m = p.qs[q].m;
        const int nh = p.n_hyp[q];
        const int64_t slot_base = 4 * p.wq[q].s_begin;
        const float tau2 = d.tau2;

        // pose h as 12 projection coefficients (K [R | t] rows), each duplicated
        // into both halves of a packed pair
        uint64_t P[HT][12];
#pragma unroll
        for (int h = 0; h < HT; ++h) {
            const int j = tile * TH + h * THREADS + tid;
            float c12[12];
            if (j < nh) {
                const int id = d.compact[j];
                const PoseF ps = d.slots[id - slot_base];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    c12[c] = d.fx * ps.R[c] + d.cx * ps.R[6 + c];
                    c12[4 + c] = d.fy * ps.R[3 + c] + d.cy * ps.R[6 + c];
                    c12[8 + c] = ps.R[6 + c];
                }
                c12[3] = d.fx * ps.t[0] + d.cx * ps.t[2];
                c12[7] = d.fy * ps.t[1] + d.cy * ps.t[2];
                c12[11] = ps.t[2];
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) c12[c] = 0.f;
            }
#pragma unroll
            for (int c = 0; c < 12; ++c) P[h][c] = f2_pack(c12[c], c12[c]);
        }
        // this CTA's share of the record pairs
        const int m2 = (m + 1) >> 1;
        const int c0 = static_cast<int>(static_cast<int64_t>(m2) * rank / CS);
        const int c1 = static_cast<int>(static_cast<int64_t>(m2) * (rank + 1) / CS);
        const int nwin = (c1 - c0 + kWinPairs - 1) / kWinPairs;
        float acc[HT];
        int cnt[HT];
#pragma unroll
        for (int h = 0; h < HT; ++h) { acc[h] = 0.f; cnt[h] = 0; }

        for (int w = 0; w < nwin; ++w) {
            const int w0 = c0 + w * kWinPairs;
            const int npair_w = min(kWinPairs, c1 - w0);
            const int nch = (npair_w + kChunkPairs - 1) / kChunkPairs;
            const bool reuse = (nwin == 1 && q == loaded_q && w0 == loaded_w0 && npair_w == loaded_n);
            if (!reuse) {
                if (nwin > 1) __syncthreads();  // all threads done with the previous window
                if (tid == 0) {
                    for (int c = 0; c < nch; ++c) {
                        const int np = min(kChunkPairs, npair_w - c * kChunkPairs);
                        const uint32_t bytes = static_cast<uint32_t>(np * sizeof(ScorePair));
                        mbar_arrive_expect_tx(&bar[c], bytes);
                        bulk_g2s(buf + c * kChunkPairs, d.subset + w0 + c * kChunkPairs, bytes, &bar[c]);
                    }
                }
                if (nwin == 1) { loaded_q = q; loaded_w0 = w0; loaded_n = npair_w; }
                else loaded_q = -1;
            }
            for (int c = 0; c < nch; ++c) {
                if (!reuse) {
                    mbar_wait_bounded(&bar[c], (phases >> c) & 1u, p.err);
                    phases ^= (1u << c);
                }
                const int np = min(kChunkPairs, npair_w - c * kChunkPairs);
                const float4* rec = reinterpret_cast<const float4*>(buf + c * kChunkPairs);
                // partial sums of the chunk: even records and odd records, each in order
                float pe[HT], po[HT];
#pragma unroll
                for (int h = 0; h < HT; ++h) { pe[h] = 0.f; po[h] = 0.f; }
#pragma unroll UNR
                for (int k = 0; k < np; ++k) {
                    const float4 A = rec[3 * k];      // X0 X1 Y0 Y1
                    const float4 B = rec[3 * k + 1];  // Z0 Z1 w0 w1
                    const float4 E = rec[3 * k + 2];  // -x0 -x1 -y0 -y1
                    const uint64_t X2 = f2_pack(A.x, A.y), Y2 = f2_pack(A.z, A.w), Z2 = f2_pack(B.x, B.y);
#pragma unroll
                    for (int h = 0; h < HT; ++h) {
                        // the projection of both records: 9 packed FMAs
                        const uint64_t zu = f2_fma(P[h][0], X2, f2_fma(P[h][1], Y2, f2_fma(P[h][2], Z2, P[h][3])));
                        const uint64_t zv = f2_fma(P[h][4], X2, f2_fma(P[h][5], Y2, f2_fma(P[h][6], Z2, P[h][7])));
                        const uint64_t zz = f2_fma(P[h][8], X2, f2_fma(P[h][9], Y2, f2_fma(P[h][10], Z2, P[h][11])));
                        float z0, z1;
                        f2_unpack(zz, z0, z1);
                        // z <= 0 (or NaN) -> 1/0 = inf -> r2 inf/NaN -> min(., tau2) = tau2
                        const float i0 = rcp_approx(fmaxf(z0, 0.0f)), i1 = rcp_approx(fmaxf(z1, 0.0f));
                        // residuals of both records packed again (E holds -x0 -x1 -y0 -y1 as pairs)
                        const uint64_t iz2 = f2_pack(i0, i1);
                        const uint64_t du2 = f2_fma(zu, iz2, f2_pack(E.x, E.y));
                        const uint64_t dv2 = f2_fma(zv, iz2, f2_pack(E.z, E.w));
                        float r0, r1;
                        f2_unpack(f2_fma(du2, du2, f2_mul(dv2, dv2)), r0, r1);
                        pe[h] = fmaf(B.z, fminf(r0, tau2), pe[h]);
                        po[h] = fmaf(B.w, fminf(r1, tau2), po[h]);
                        if (COUNT) cnt[h] += ((r0 < tau2) ? 1 : 0) + ((r1 < tau2) ? 1 : 0);
                    }
                }
#pragma unroll
                for (int h = 0; h < HT; ++h) acc[h] += pe[h] + po[h];
            }
        }

        // combine the CS partial sums of each pose through distributed shared memory
#pragma unroll
        for (int h = 0; h < HT; ++h) {
            s_part[h * THREADS + tid] = acc[h];
            if (COUNT) s_cnt[h * THREADS + tid] = cnt[h];
        }
        cluster.sync();
        const int per = TH / CS;
        for (int e = rank * per + tid; e < (rank + 1) * per; e += THREADS) {
            float sc = 0.f;
            int ct = 0;
            for (int r = 0; r < CS; ++r) {
                sc += cluster.map_shared_rank(s_part, r)[e];
                if (COUNT) ct += cluster.map_shared_rank(s_cnt, r)[e];
            }
            const int j = tile * TH + e;
            const bool valid = j < nh;
            uint32_t id = 0xffffffffu, rd = 0xffffffffu, sb = 0xffffffffu;
            if (valid) {
                id = static_cast<uint32_t>(d.compact[j]);
                rd = static_cast<uint32_t>((id >> 2) / static_cast<uint32_t>(d.batch));
                sb = __float_as_uint(sc);
                if (d.score_by_id) d.score_by_id[id - slot_base] = sc;
                if (COUNT && d.count_by_id) d.count_by_id[id - slot_base] = ct;
            }
            // per round, the minimum (score bits, pose id) of the warp, then one atomic
            unsigned long long kv = valid ? ((static_cast<unsigned long long>(sb) << 32) | id) : ~0ull;
            bool pending = valid;
            while (__any_sync(0xffffffffu, pending)) {
                const int first = __ffs(__ballot_sync(0xffffffffu, pending)) - 1;
                const uint32_t r0 = __shfl_sync(0xffffffffu, rd, first);
                unsigned long long v = (pending && rd == r0) ? kv : ~0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
                    v = u < v ? u : v;
                }
                if (lane == first) atomicMin(reinterpret_cast<unsigned long long*>(&d.round_best[r0]), v);
                if (rd == r0) pending = false;
            }
        }
        // s_part is rewritten only after the next item's first cluster barrier,
        // which every CTA reaches after finishing the reads above; the subset
        // buffer is rewritten only after both item barriers.
        }  // scored tile
        if constexpr (FUSED) {
            // the item is complete in every CTA (its minima are visible device-wide)
            __threadfence();
            cluster.sync();
            if (rank == 0 && threadIdx.x == 0) {
                const int items_q = p.tile_prefix[q + 1] - p.tile_prefix[q];
                const int old = atomicAdd(&p.qdone[q], 1);
                s_last = (old + 1 == items_q) ? 1 : 0;
            }
            cluster.sync();
            const int last = *cluster.map_shared_rank(&s_last, 0);
            if (last && !d.lo_fp64) {
                __threadfence();
                if (threadIdx.x == 0) {
                    S_rep.stg = nullptr;
                    S_rep.stg_cap = 0;
                }
                replay_query<float, THREADS>(S_rep, d, p.qs + q, p.wq[q], cluster, CS, rank);
            }
        }
    }
}

// ============================================================================
// bf16-packed scoring (option score_bf16)
// ============================================================================
// k_setup_bf16 (one CTA per query, after k_setup): the bounding box of the
// subset's records (the zero-weight padding record of an odd subset
// included) gives the centre c (its midpoint) and the scale s (the smallest
// power of two >= its half extent), so |X'| = |X - c| / s <= 1 per
// coordinate; X' is rounded to bf16 (relative error <= 2^-9 of |X'| <= 1).
// Reconstruction error per world coordinate: |X - c - s bf16(fl(X - c) / s)|
// <= 2^-24 s + 2^-9 s = e.  The header also holds max |x|, max |y| of the
// observed pixels and the sum of the weights.
__global__ void __launch_bounds__(512) k_setup_bf16(const QueryDesc* qd, const QueryState* qs, const int32_t* init_list) {
    const int q = init_list ? init_list[blockIdx.x] : blockIdx.x;
    const QueryDesc& d = qd[q];
    if (!d.subset_b) return;
    const int m = qs[q].m, m2 = (m + 1) >> 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float xm = 0.f, ym = 0.f, ws = 0.f;
    for (int k2 = tid; k2 < m2; k2 += 512) {
        const ScorePair& P = d.subset[k2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            lo[0] = fminf(lo[0], P.X[l]); hi[0] = fmaxf(hi[0], P.X[l]);
            lo[1] = fminf(lo[1], P.Y[l]); hi[1] = fmaxf(hi[1], P.Y[l]);
            lo[2] = fminf(lo[2], P.Z[l]); hi[2] = fmaxf(hi[2], P.Z[l]);
            xm = fmaxf(xm, fabsf(P.nx[l]));
            ym = fmaxf(ym, fabsf(P.ny[l]));
            ws += P.w[l];
        }
    }
    __shared__ float s_red[16][9];
    __shared__ ScoreHeadB s_head;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, o));
        ym = fmaxf(ym, __shfl_xor_sync(0xffffffffu, ym, o));
        ws += __shfl_xor_sync(0xffffffffu, ws, o);
    }
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) { s_red[warp][a] = lo[a]; s_red[warp][3 + a] = hi[a]; }
        s_red[warp][6] = xm; s_red[warp][7] = ym; s_red[warp][8] = ws;
    }
    __syncthreads();
    if (tid == 0) {
        float L[3], Hh[3], X = 0.f, Y = 0.f, W = 0.f;
        for (int a = 0; a < 3; ++a) { L[a] = s_red[0][a]; Hh[a] = s_red[0][3 + a]; }
        X = s_red[0][6]; Y = s_red[0][7]; W = s_red[0][8];
        for (int w = 1; w < 16; ++w) {
            for (int a = 0; a < 3; ++a) { L[a] = fminf(L[a], s_red[w][a]); Hh[a] = fmaxf(Hh[a], s_red[w][3 + a]); }
            X = fmaxf(X, s_red[w][6]); Y = fmaxf(Y, s_red[w][7]); W += s_red[w][8];
        }
        ScoreHeadB h;
        float half = 0.f;
        for (int a = 0; a < 3; ++a) {
            if (!(L[a] <= Hh[a])) { L[a] = 0.f; Hh[a] = 0.f; }  // empty subset
            h.c[a] = 0.5f * L[a] + 0.5f * Hh[a];
            half = fmaxf(half, fmaxf(Hh[a] - h.c[a], h.c[a] - L[a]));
        }
        // smallest power of two >= half (1 + 2^-16), at least 2^-40
        float sc = 0x1p-40f;
        while (sc < half * (1.0f + 0x1p-16f)) sc *= 2.0f;
        h.s = sc;
        h.e = sc * (0x1p-9f + 0x1p-23f);
        h.xmax = X;
        h.ymax = Y;
        h.wsum = W;
        s_head = h;
        *reinterpret_cast<ScoreHeadB*>(d.subset_b) = h;
    }
    __syncthreads();
    const ScoreHeadB h = s_head;
    const float inv_s = 1.0f / h.s;  // a power of two: exact
    for (int k2 = tid; k2 < m2; k2 += 512) {
        const ScorePair& P = d.subset[k2];
        ScorePairB b;
        b.X2 = bf16_pair((P.X[0] - h.c[0]) * inv_s, (P.X[1] - h.c[0]) * inv_s);
        b.Y2 = bf16_pair((P.Y[0] - h.c[1]) * inv_s, (P.Y[1] - h.c[1]) * inv_s);
        b.Z2 = bf16_pair((P.Z[0] - h.c[2]) * inv_s, (P.Z[1] - h.c[2]) * inv_s);
        b.pad = 0u;
        b.nx[0] = P.nx[0]; b.nx[1] = P.nx[1];
        b.ny[0] = P.ny[0]; b.ny[1] = P.ny[1];
        d.subset_b[1 + k2] = b;
    }
}

// k_score_bf16: the persistent, cluster-split scoring of k_score (same work
// queue, same shares of the subset per CTA), with the shares held as
// bf16-packed record pairs (32 B instead of 48 B) and every (pose, record)
// pair first classified from them.  Per pose, folded with the header,
// F = [s P_{0:3} | P (c, 1)] gives the homogeneous residual
// d = (F_u X' - x F_z X', F_v X' - y F_z X') and depth z = F_z X'.  Against
// the FP32 values of the same pair they differ by at most
// A_u = (|P_u|_1 + xmax |P_z|_1) e + rho M_u..., bz = |P_z|_1 e + rho M_z
// (e: the header's reconstruction bound, rho M: FP32 rounding of both
// evaluations), so the pair is surely an outlier of the FP32 scoring (r >= tau)
// if z <= -bz, or if z > bz and |d| >= tau_e (z + bz) + |A| (triangle
// inequality; tau_e = tau plus a 1e-3 px margin).  Such a pair contributes
// w tau^2 and no inlier; every other pair is rescored in FP32 from the FP32
// record (global memory, L1) and the unfolded pose (shared memory) with the
// FP32 kernel's arithmetic, so the inlier counts equal the FP32 kernel's and
// the scores agree with them up to FP32 summation order:
// score = tau^2 sum(w) + sum over rescored pairs of w (min(r^2, tau^2) - tau^2).
constexpr int kBfThreads = 128, kBfHT = 4, kBfTile = kBfThreads * kBfHT;
static_assert(kBfTile <= kMaxTileHyps && kBfTile % kScoreCluster == 0, "tile size");

static size_t score_bf16_smem_bytes() {
    return sizeof(ScorePairB) * kWinPairs + sizeof(float) * 12 * kBfTile + sizeof(float) * kBfTile +
           sizeof(int) * kBfTile;
}

template <bool COUNT>
__global__ void __launch_bounds__(kBfThreads, 1) k_score_bf16(const __grid_constant__ ScoreParams p) {
    constexpr int THREADS = kBfThreads, HT = kBfHT, TH = kBfTile;
    extern __shared__ __align__(128) unsigned char smem[];
    ScorePairB* buf = reinterpret_cast<ScorePairB*>(smem);
    float* s_pose = reinterpret_cast<float*>(buf + kWinPairs);  // unfolded pose coefficient k of pose e at [k * TH + e]
    float* s_part = s_pose + 12 * TH;
    int* s_cnt = reinterpret_cast<int*>(s_part + TH);
    __shared__ __align__(8) uint64_t bar[kWinChunks];
    __shared__ int s_item;

    cg::cluster_group cluster = cg::this_cluster();
    const int CS = static_cast<int>(cluster.num_blocks());
    const int rank = static_cast<int>(cluster.block_rank());
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        for (int c = 0; c < kWinChunks; ++c) mbar_init(&bar[c], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t phases = 0u;
    int loaded_q = -1, loaded_w0 = -1, loaded_n = -1;
    const int total_tiles = p.tile_prefix[p.nq];
    unsigned long long rescored = 0ull;
    constexpr float kRho = 0x1p-20f;

    for (;;) {
        if (rank == 0 && tid == 0) s_item = static_cast<int>(atomicAdd(p.work_counter, 1u));
        cluster.sync();
        const int item = *cluster.map_shared_rank(&s_item, 0);
        cluster.sync();
        if (item >= total_tiles) break;
        int lo = 0, hi = p.nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.tile_prefix[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int q = lo;
        const int tile = item - p.tile_prefix[q];
        const QueryDesc& d = p.qd[q];
        if (tile >= p.ntiles[q]) continue;
        const int m = p.qs[q].m;
        const int nh = p.n_hyp[q];
        const int64_t slot_base = 4 * p.wq[q].s_begin;
        const float tau2 = d.tau2;
        const ScoreHeadB H = *reinterpret_cast<const ScoreHeadB*>(d.subset_b);
        const float cmax = fmaxf(fabsf(H.c[0]), fmaxf(fabsf(H.c[1]), fabsf(H.c[2])));
        const float tau_e = (sqrtf(tau2) * (1.0f + kRho) + 1e-3f + kRho * fmaxf(H.xmax, H.ymax)) * (1.0f + kRho);
        const uint64_t TAU = f2_pack(tau_e, tau_e);

        // poses: folded coefficients (packed, duplicated), the bounds, and the
        // unfolded coefficients in shared memory for the FP32 rescoring
        uint64_t F[HT][12], CST[HT];
        float BZ[HT];
#pragma unroll
        for (int h = 0; h < HT; ++h) {
            const int e = h * THREADS + tid;
            const int j = tile * TH + e;
            float c12[12];
            if (j < nh) {
                const int id = d.compact[j];
                const PoseF ps = d.slots[id - slot_base];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    c12[c] = d.fx * ps.R[c] + d.cx * ps.R[6 + c];
                    c12[4 + c] = d.fy * ps.R[3 + c] + d.cy * ps.R[6 + c];
                    c12[8 + c] = ps.R[6 + c];
                }
                c12[3] = d.fx * ps.t[0] + d.cx * ps.t[2];
                c12[7] = d.fy * ps.t[1] + d.cy * ps.t[2];
                c12[11] = ps.t[2];
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) c12[c] = 0.f;
            }
            float N[3], M[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float* P = c12 + 4 * r;
                N[r] = fabsf(P[0]) + fabsf(P[1]) + fabsf(P[2]);
                M[r] = N[r] * (cmax + H.s) + fabsf(P[3]);
                const float f3 = fmaf(P[0], H.c[0], fmaf(P[1], H.c[1], fmaf(P[2], H.c[2], P[3])));
#pragma unroll
                for (int k = 0; k < 3; ++k) F[h][4 * r + k] = f2_pack(H.s * P[k], H.s * P[k]);
                F[h][4 * r + 3] = f2_pack(f3, f3);
            }
            const float Au = (N[0] + H.xmax * N[2]) * H.e + kRho * (M[0] + H.xmax * M[2]);
            const float Av = (N[1] + H.ymax * N[2]) * H.e + kRho * (M[1] + H.ymax * M[2]);
            const float A = sqrtf(Au * Au + Av * Av) * (1.0f + kRho);
            BZ[h] = N[2] * H.e + kRho * M[2];
            const float cst = (tau_e * BZ[h] + A) * (1.0f + kRho);
            CST[h] = f2_pack(cst, cst);
#pragma unroll
            for (int k = 0; k < 12; ++k) s_pose[k * TH + e] = c12[k];
        }
        __syncthreads();  // s_pose of this item (rewritten only after the next item's cluster barriers)

        const int m2 = (m + 1) >> 1;
        const int c0 = static_cast<int>(static_cast<int64_t>(m2) * rank / CS);
        const int c1 = static_cast<int>(static_cast<int64_t>(m2) * (rank + 1) / CS);
        const int nwin = (c1 - c0 + kWinPairs - 1) / kWinPairs;
        float acc[HT];
        int cnt[HT];
#pragma unroll
        for (int h = 0; h < HT; ++h) { acc[h] = 0.f; cnt[h] = 0; }

        for (int w = 0; w < nwin; ++w) {
            const int w0 = c0 + w * kWinPairs;
            const int npair_w = min(kWinPairs, c1 - w0);
            const int nch = (npair_w + kChunkPairs - 1) / kChunkPairs;
            const bool reuse = (nwin == 1 && q == loaded_q && w0 == loaded_w0 && npair_w == loaded_n);
            if (!reuse) {
                if (nwin > 1) __syncthreads();
                if (tid == 0) {
                    for (int c = 0; c < nch; ++c) {
                        const int np = min(kChunkPairs, npair_w - c * kChunkPairs);
                        const uint32_t bytes = static_cast<uint32_t>(np * sizeof(ScorePairB));
                        mbar_arrive_expect_tx(&bar[c], bytes);
                        bulk_g2s(buf + c * kChunkPairs, d.subset_b + 1 + w0 + c * kChunkPairs, bytes, &bar[c]);
                    }
                }
                if (nwin == 1) { loaded_q = q; loaded_w0 = w0; loaded_n = npair_w; }
                else loaded_q = -1;
            }
            for (int c = 0; c < nch; ++c) {
                if (!reuse) {
                    mbar_wait_bounded(&bar[c], (phases >> c) & 1u, p.err);
                    phases ^= (1u << c);
                }
                const int np = min(kChunkPairs, npair_w - c * kChunkPairs);
                const uint4* rq = reinterpret_cast<const uint4*>(buf + c * kChunkPairs);
                const float4* rf = reinterpret_cast<const float4*>(buf + c * kChunkPairs);
                const float4* gsub = reinterpret_cast<const float4*>(d.subset + w0 + c * kChunkPairs);
                for (int k = 0; k < np; ++k) {
                    const uint4 Q = rq[2 * k];
                    const float4 E = rf[2 * k + 1];  // -x0 -x1 -y0 -y1
                    const uint64_t X2 = f2_pack(__uint_as_float(Q.x << 16), __uint_as_float(Q.x & 0xffff0000u));
                    const uint64_t Y2 = f2_pack(__uint_as_float(Q.y << 16), __uint_as_float(Q.y & 0xffff0000u));
                    const uint64_t Z2 = f2_pack(__uint_as_float(Q.z << 16), __uint_as_float(Q.z & 0xffff0000u));
                    const uint64_t NX = f2_pack(E.x, E.y), NY = f2_pack(E.z, E.w);
#pragma unroll
                    for (int h = 0; h < HT; ++h) {
                        const uint64_t zu = f2_fma(F[h][0], X2, f2_fma(F[h][1], Y2, f2_fma(F[h][2], Z2, F[h][3])));
                        const uint64_t zv = f2_fma(F[h][4], X2, f2_fma(F[h][5], Y2, f2_fma(F[h][6], Z2, F[h][7])));
                        const uint64_t zz = f2_fma(F[h][8], X2, f2_fma(F[h][9], Y2, f2_fma(F[h][10], Z2, F[h][11])));
                        const uint64_t du = f2_fma(NX, zz, zu), dv = f2_fma(NY, zz, zv);
                        const uint64_t T = f2_fma(TAU, zz, CST[h]);
                        float z0, z1, d0, d1, t0, t1;
                        f2_unpack(zz, z0, z1);
                        f2_unpack(f2_fma(du, du, f2_mul(dv, dv)), d0, d1);
                        f2_unpack(f2_mul(T, T), t0, t1);
                        const float bz = BZ[h];
                        const bool out0 = (z0 <= -bz) || (z0 > bz && d0 >= t0);
                        const bool out1 = (z1 <= -bz) || (z1 > bz && d1 >= t1);
                        if (!(out0 && out1)) {
                            // FP32 rescoring with the FP32 kernel's arithmetic
                            const int e = h * THREADS + tid;
                            float P[12];
#pragma unroll
                            for (int a = 0; a < 12; ++a) P[a] = s_pose[a * TH + e];
                            const float4 A4 = __ldg(gsub + 3 * k), B4 = __ldg(gsub + 3 * k + 1), E4 = __ldg(gsub + 3 * k + 2);
#pragma unroll
                            for (int l = 0; l < 2; ++l) {
                                if (l == 0 ? out0 : out1) continue;
                                const float X = l ? A4.y : A4.x, Y = l ? A4.w : A4.z, Z = l ? B4.y : B4.x;
                                const float wl = l ? B4.w : B4.z, nx = l ? E4.y : E4.x, ny = l ? E4.w : E4.z;
                                const float u_ = fmaf(P[0], X, fmaf(P[1], Y, fmaf(P[2], Z, P[3])));
                                const float v_ = fmaf(P[4], X, fmaf(P[5], Y, fmaf(P[6], Z, P[7])));
                                const float z_ = fmaf(P[8], X, fmaf(P[9], Y, fmaf(P[10], Z, P[11])));
                                const float iz = rcp_approx(fmaxf(z_, 0.0f));
                                const float ru = fmaf(u_, iz, nx), rv = fmaf(v_, iz, ny);
                                const float r2 = fmaf(ru, ru, rv * rv);
                                acc[h] = fmaf(wl, fminf(r2, tau2) - tau2, acc[h]);
                                if (COUNT) cnt[h] += (r2 < tau2) ? 1 : 0;
                                ++rescored;
                            }
                        }
                    }
                }
            }
        }

#pragma unroll
        for (int h = 0; h < HT; ++h) {
            s_part[h * THREADS + tid] = acc[h];
            if (COUNT) s_cnt[h * THREADS + tid] = cnt[h];
        }
        cluster.sync();
        const int per = TH / CS;
        for (int e = rank * per + tid; e < (rank + 1) * per; e += THREADS) {
            float sc = 0.f;
            int ct = 0;
            for (int r = 0; r < CS; ++r) {
                sc += cluster.map_shared_rank(s_part, r)[e];
                if (COUNT) ct += cluster.map_shared_rank(s_cnt, r)[e];
            }
            sc = fmaf(tau2, H.wsum, sc);
            const int j = tile * TH + e;
            const bool valid = j < nh;
            uint32_t id = 0xffffffffu, rd = 0xffffffffu, sb = 0xffffffffu;
            if (valid) {
                id = static_cast<uint32_t>(d.compact[j]);
                rd = static_cast<uint32_t>((id >> 2) / static_cast<uint32_t>(d.batch));
                sb = __float_as_uint(sc);
                if (d.score_by_id) d.score_by_id[id - slot_base] = sc;
                if (COUNT && d.count_by_id) d.count_by_id[id - slot_base] = ct;
            }
            unsigned long long kv = valid ? ((static_cast<unsigned long long>(sb) << 32) | id) : ~0ull;
            bool pending = valid;
            while (__any_sync(0xffffffffu, pending)) {
                const int first = __ffs(__ballot_sync(0xffffffffu, pending)) - 1;
                const uint32_t r0 = __shfl_sync(0xffffffffu, rd, first);
                unsigned long long v = (pending && rd == r0) ? kv : ~0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
                    v = u < v ? u : v;
                }
                if (lane == first) atomicMin(reinterpret_cast<unsigned long long*>(&d.round_best[r0]), v);
                if (rd == r0) pending = false;
            }
        }
    }
    if (p.rescored) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rescored += __shfl_xor_sync(0xffffffffu, rescored, o);
        if (lane == 0 && rescored) atomicAdd(p.rescored, rescored);
    }
}

// ============================================================================
// k_score_tc: hypothesis scoring with the projection on the tensor cores
// ============================================================================
// The projections of a tile of 128 poses on a block of NB subset records are
// three matrix products (rows K [R | t]_u, _v, _z of the poses times the
// records' (X, Y, Z, 1)).  They run as tcgen05.mma with K = 24 (of 32): both
// operands are split into three pieces (pose coefficient a = a0 + a1 + a2,
// record component b = b0 + b1 + b2; bf16 pieces for kind::f16, two K steps
// of 16, or TF32 pieces for kind::tf32, three K steps of 8) and the six piece
// products that carry the FP32 value (a0 b0, a0 b1, a1 b0, a0 b2, a1 b1,
// a2 b0) are the K lanes; every piece product is exact in FP32, so the
// accumulator holds the FP32 projection to a few FP32 ulps.
// The FP32 accumulators land in TMEM; the epilogue warps (thread = pose =
// TMEM lane) read them back with tcgen05.ld and do the rest of the cost in
// FP32: reciprocal of the depth (z <= 0 or NaN -> tau^2), residual,
// truncation, weighted sum.
//
// One CTA per SM, persistent over the (query, 128-pose tile) queue; every
// CTA streams all records of its item's query (bulk copies of NB operand
// rows of 128 bytes + NB x 16 bytes of pixels and weights per block, a ring
// of stages).  Warps:
//   4 NG + 1           producer: waits for a free stage, bulk copies into it
//   4 NG               TMEM allocation; the converged warp walks the blocks,
//                      one elected lane issues the block's MMAs (3 rows x K
//                      steps) into a free accumulator buffer and commits them
//                      to the buffer's mbarrier
//   0 .. 4 NG - 1      epilogue: NG groups of four warps (warp w reads TMEM
//                      lanes 32 (w mod 4) ..); group g takes records g NB/NG ..
//                      (g + 1) NB/NG - 1 of every block, frees the buffer once
//                      it has loaded them and the stage once it has used the
//                      pixels; warps 0-3 also write the pose rows of each item
// Per pose, each group sums its records in block order (within its part of
// a block the even and the odd records separately, then even + odd), and the
// score adds the group sums in group order: independent of timing and of the
// grid.
constexpr int kTcPoses = 128;
constexpr uint32_t kTcCols = 512;
constexpr uint32_t kTcATile = 128 * 128;  // one pose-row operand in shared memory: 128 rows of 128 bytes

// NB records per block, NG epilogue groups of 4 warps; every group reads NB / NG
// columns (records) of every block
template <int NB, int NG>
struct TcShape {
    static constexpr int kThreads = NG * 128 + 64;          // + the MMA warp and the producer warp
    static constexpr int kStages = NB <= 32 ? 16 : (NB <= 80 ? 8 : 6);
    static constexpr int kBufs = 512 / (3 * NB);           // accumulator buffers of 3 x NB TMEM columns
    static constexpr int kCols = NB / NG;                  // records of a block per group
    static_assert(kCols % 16 == 0 && kBufs >= 1, "shape");
    static constexpr uint32_t kBStage = NB * 128;
    static constexpr uint32_t kEStage = NB * 16;
    // at least 116 KB, so that one CTA holds an SM (and all of its TMEM)
    static constexpr size_t kSmemNeed = 1024 + 3 * kTcATile + kStages * (kBStage + kEStage) + NG * kTcPoses * 8 +
                                        (2 * kStages + 2 * kBufs) * 8 + 16;
    static constexpr size_t kSmem = kSmemNeed > 116 * 1024 ? kSmemNeed : 116 * 1024;
};
static_assert(kTcBlock % 128 == 0 && kTcBlock % 80 == 0, "record padding covers every block size");

template <int NB, int NG, bool BF, bool COUNT>
__global__ void __launch_bounds__(TcShape<NB, NG>::kThreads, 1) k_score_tc(const __grid_constant__ ScoreParams p) {
    using TS = TcShape<NB, NG>;
    constexpr int S = TS::kStages, NBUF = TS::kBufs;
    constexpr int KSTEPS = BF ? 2 : 3;  // 32-byte K steps of one MMA each
    constexpr int WMMA = 4 * NG, WPROD = 4 * NG + 1;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = smem;                                   // rows u, v, z: 3 x 16 KB
    unsigned char* sB = sA + 3 * kTcATile;                      // ring of record operand blocks
    float4* sE = reinterpret_cast<float4*>(sB + S * TS::kBStage);  // ring of pixel / weight blocks
    float* s_part = reinterpret_cast<float*>(sE + S * (TS::kEStage / 16));  // [NG][128] per group
    int* s_cntp = reinterpret_cast<int*>(s_part + NG * kTcPoses);          // [NG][128]
    uint64_t* full = reinterpret_cast<uint64_t*>(s_cntp + NG * kTcPoses);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NBUF;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + NBUF);
    int* s_item = reinterpret_cast<int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            // every epilogue warp, once done with the block: it waited for its MMAs and read its pixels
            mbar_init(&empty[st], 4 * NG);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4 * NG);
        }
        mbar_fence_init();
    }
    if (warp == WMMA) {
        tmem_alloc(tmem_slot, kTcCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int total_tiles = p.tile_prefix[p.nq];
    uint32_t base = 0;  // record blocks of the earlier items of this CTA (ring and buffer positions)

    for (;;) {
        if (tid == 0) *s_item = static_cast<int>(atomicAdd(p.work_counter, 1u));
        __syncthreads();  // also: every MMA of the previous item has completed (its epilogue consumed them)
        const int item = *s_item;
        if (item >= total_tiles) break;
        int lo = 0, hi = p.nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.tile_prefix[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int q = lo;
        const int tile = item - p.tile_prefix[q];
        const QueryDesc& d = p.qd[q];
        const bool active = tile < p.ntiles[q];
        const int m = active ? p.qs[q].m : 0;
        const int nh = p.n_hyp[q];
        const int nblk = (m + NB - 1) / NB;
        const int64_t slot_base = 4 * p.wq[q].s_begin;

        if (active && warp < 4) {
            // pose rows of this item: thread tid writes pose tile * 128 + tid
            const int j = tile * kTcPoses + tid;
            float c12[12];
            if (j < nh) {
                const PoseF ps = d.slots[d.compact[j] - slot_base];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    c12[c] = d.fx * ps.R[c] + d.cx * ps.R[6 + c];
                    c12[4 + c] = d.fy * ps.R[3 + c] + d.cy * ps.R[6 + c];
                    c12[8 + c] = ps.R[6 + c];
                }
                c12[3] = d.fx * ps.t[0] + d.cx * ps.t[2];
                c12[7] = d.fy * ps.t[1] + d.cy * ps.t[2];
                c12[11] = ps.t[2];
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) c12[c] = 0.f;
            }
            const int sw = tid & 7;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                uint4 ch[8];
                tc_operand_row(c12 + 4 * r, BF, true, ch);
                uint4* row = reinterpret_cast<uint4*>(sA + r * kTcATile + (tid >> 3) * 1024 + (tid & 7) * 128);
#pragma unroll
                for (int c = 0; c < 2 * KSTEPS; ++c) row[c ^ sw] = ch[c];  // the chunks the K steps read
            }
            // the generic-proxy writes become visible to the tensor core's reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.arrive 2, 160;" ::: "memory");
        } else if (active && warp == WMMA) {
            // the whole warp walks the blocks (it stays converged); lane 0 issues
            asm volatile("bar.sync 2, 160;" ::: "memory");  // pose rows written
            constexpr uint32_t idesc = BF ? umma_idesc_bf16(kTcPoses, NB) : umma_idesc_tf32(kTcPoses, NB);
            // descriptor start addresses advance by byte offset >> 4 (fields stay below 2^14)
            const uint64_t adesc = umma_desc_k_sw128(smem_u32(sA)), bdesc = umma_desc_k_sw128(smem_u32(sB));
            for (int b = 0; b < nblk; ++b) {
                const uint32_t gb = base + b;
                const uint32_t st = gb % S, buf = gb % NBUF;
                mbar_wait_bounded(&tempty[buf], ((gb / NBUF) & 1u) ^ 1u, p.err);
                mbar_wait_bounded(&full[st], (gb / S) & 1u, p.err);
                tc_fence_after();
                const uint64_t bd0 = bdesc + ((st * TS::kBStage) >> 4);
                const uint32_t d0 = tmem_base + buf * 3 * NB;
                if (elect_one()) {
#pragma unroll
                    for (int kk = 0; kk < KSTEPS; ++kk) {
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            const uint64_t ad = adesc + ((r * kTcATile + kk * 32) >> 4);
                            const uint64_t bd = bd0 + ((kk * 32) >> 4);
                            if constexpr (BF) umma_bf16(d0 + r * NB, ad, bd, idesc, kk > 0 ? 1u : 0u);
                            else umma_tf32(d0 + r * NB, ad, bd, idesc, kk > 0 ? 1u : 0u);
                        }
                    }
                    // accumulators ready; the stage is freed by the epilogue, which waits for this
                    umma_commit(&tfull[buf]);
                }
                __syncwarp();
            }
        } else if (active && warp == WPROD) {
            for (int b = 0; b < nblk; ++b) {
                const uint32_t gb = base + b;
                const uint32_t st = gb % S;
                mbar_wait_bounded(&empty[st], ((gb / S) & 1u) ^ 1u, p.err);
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[st], TS::kBStage + TS::kEStage);
                    bulk_g2s(sB + st * TS::kBStage, d.tc_rec + static_cast<int64_t>(b) * NB * 8, TS::kBStage, &full[st]);
                    bulk_g2s(sE + st * (TS::kEStage / 16), d.tc_e + static_cast<int64_t>(b) * NB, TS::kEStage, &full[st]);
                }
                __syncwarp();
            }
        }
        if (active && warp < 4 * NG) {
            const int g = warp >> 2, wq = warp & 3;
            const float tau2 = d.tau2;
            float tot = 0.f;
            int cnt = 0;
            const uint32_t lane_addr = tmem_base + (static_cast<uint32_t>(wq * 32) << 16);
            constexpr int CW = TS::kCols;
            for (int b = 0; b < nblk; ++b) {
                const uint32_t gb = base + b;
                const uint32_t st = gb % S, buf = gb % NBUF;
                mbar_wait_bounded(&tfull[buf], (gb / NBUF) & 1u, p.err);
                tc_fence_after();
                // this group's records of the block: g * CW .. g * CW + CW - 1
                const float4* E = sE + st * (TS::kEStage / 16) + g * CW;
                uint64_t acc2 = f2_pack(0.f, 0.f);
#pragma unroll 1
                for (int h = 0; h < CW / 16; ++h) {
                    uint32_t zu[16], zv[16], zz[16];
                    const uint32_t ta = lane_addr + buf * 3 * NB + g * CW + h * 16;
                    tmem_ld_32x32b_x16_nowait(ta, zu);
                    tmem_ld_32x32b_x16_nowait(ta + NB, zv);
                    tmem_ld_32x32b_x16_nowait(ta + 2 * NB, zz);
                    tmem_wait_ld();
                    if (h == CW / 16 - 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[buf]);
                    }
                    // the pixels and weights of the block (landed with the operand rows)
                    if (h == 0) mbar_wait_bounded(&full[st], (gb / S) & 1u, p.err);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float4 e = E[16 * h + 2 * k];  // -x0 -x1 -y0 -y1
                        const float2 w = *reinterpret_cast<const float2*>(E + 16 * h + 2 * k + 1);
                        const float z0 = __uint_as_float(zz[2 * k]), z1 = __uint_as_float(zz[2 * k + 1]);
                        const float i0 = rcp_approx(fmaxf(z0, 0.0f)), i1 = rcp_approx(fmaxf(z1, 0.0f));
                        const uint64_t iz2 = f2_pack(i0, i1);
                        const uint64_t du2 = f2_fma(f2_pack(__uint_as_float(zu[2 * k]), __uint_as_float(zu[2 * k + 1])),
                                                    iz2, f2_pack(e.x, e.y));
                        const uint64_t dv2 = f2_fma(f2_pack(__uint_as_float(zv[2 * k]), __uint_as_float(zv[2 * k + 1])),
                                                    iz2, f2_pack(e.z, e.w));
                        float r0, r1;
                        f2_unpack(f2_fma(du2, du2, f2_mul(dv2, dv2)), r0, r1);
                        acc2 = f2_fma(f2_pack(w.x, w.y), f2_pack(fminf(r0, tau2), fminf(r1, tau2)), acc2);
                        if (COUNT) cnt += ((r0 < tau2) ? 1 : 0) + ((r1 < tau2) ? 1 : 0);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
                float ae, ao;
                f2_unpack(acc2, ae, ao);
                tot += ae + ao;
            }
            // partial sums by column group, added in group order
            s_part[g * kTcPoses + wq * 32 + lane] = tot;
            if (COUNT) s_cntp[g * kTcPoses + wq * 32 + lane] = cnt;
            asm volatile("bar.sync 1, %0;" ::"n"(NG * 128) : "memory");
            if (g == 0) {
                const int e = wq * 32 + lane;
                float sc = s_part[e];
                int ct = COUNT ? s_cntp[e] : 0;
#pragma unroll
                for (int c = 1; c < NG; ++c) {
                    sc += s_part[c * kTcPoses + e];
                    if (COUNT) ct += s_cntp[c * kTcPoses + e];
                }
                const int j = tile * kTcPoses + e;
                const bool valid = j < nh;
                uint32_t id = 0xffffffffu, rd = 0xffffffffu, sb = 0xffffffffu;
                if (valid) {
                    id = static_cast<uint32_t>(d.compact[j]);
                    rd = static_cast<uint32_t>((id >> 2) / static_cast<uint32_t>(d.batch));
                    sb = __float_as_uint(sc);
                    if (d.score_by_id) d.score_by_id[id - slot_base] = sc;
                    if (COUNT && d.count_by_id) d.count_by_id[id - slot_base] = ct;
                }
                // per round, the minimum (score bits, pose id) of the warp, then one atomic
                unsigned long long kv = valid ? ((static_cast<unsigned long long>(sb) << 32) | id) : ~0ull;
                bool pending = valid;
                while (__any_sync(0xffffffffu, pending)) {
                    const int first = __ffs(__ballot_sync(0xffffffffu, pending)) - 1;
                    const uint32_t r0 = __shfl_sync(0xffffffffu, rd, first);
                    unsigned long long v = (pending && rd == r0) ? kv : ~0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
                        v = u < v ? u : v;
                    }
                    if (lane == first) atomicMin(reinterpret_cast<unsigned long long*>(&d.round_best[r0]), v);
                    if (rd == r0) pending = false;
                }
            }
        }
        base += static_cast<uint32_t>(nblk);
    }
    // every MMA completed before the epilogue read its accumulator
    tc_fence_before();
    __syncthreads();
    if (warp == WMMA) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTcCols);
    }
}

// ============================================================================
// k_score_tcr: the same products with the records on the MMA's M side
// ============================================================================
// Transposed form of k_score_tc: one MMA (M = 128 records of a block, N = 48 NG
// = the u, v and z rows of 16 NG poses, bf16 split pieces as above) per K
// step, so a block takes KSTEPS MMAs instead of 3 KSTEPS.  TMEM lane =
// record, column = (row, pose): column r 16 NG + p of a 256-column
// accumulator buffer (two buffers).  An epilogue thread owns one record of
// every block and keeps running sums for the 16 poses of its group; its
// pixel and weight come from global memory (L2), loaded one block ahead, so
// the epilogue waits only for the accumulators.  The MMA's commit frees the
// ring stage of the record rows.
// The cost of a (pose, record) pair is w tau^2 min(r^2 / tau^2, 1): the u and
// v rows of the pose are scaled by 1 / tau and the pixel by -1 / tau, so that
// the residual components come out divided by tau and one saturating FMA
// (clamp to [0, 1]) gives min(r^2 / tau^2, 1).  Points at or behind the
// camera (z <= 0, reciprocal +inf) must cost tau^2: the u and v rows carry
// 2^-100 in K lane 24 against a 1 in the record rows, so that u and v are
// never exactly 0 there and the scaled residual is infinite (saturates to 1)
// rather than 0 x inf = NaN (which a saturating FMA turns into 0).  The term
// is far below one FP32 ulp of any projection in front of the camera.
// Subset padding rows (all zero, weight 0) add 0.
// At the end of the item the sums are reduced across the 32 lanes of each
// warp (halving exchanges: 8 + 4 + 2 + 1 + 1 shuffles for 16 poses) and
// across the group's four warps in warp order.  Per pose the summation order
// is fixed by the record's position in the block and the block order:
// independent of timing and of the grid.
// Warps: 4 NG epilogue warps (NG groups of 16 poses; warp w reads TMEM lanes
// 32 (w mod 4) ..), the MMA warp, the producer warp; items are (query,
// 16 NG-pose tile).
constexpr int kTcrRecs = 128;                      // records per block (M)
constexpr int kTcrStages = 8;                      // ring of record operand blocks
constexpr uint32_t kTcrRStage = kTcrRecs * 128;    // record operand rows of a block
static_assert(kTcBlock % kTcrRecs == 0, "record padding covers the block size");

// NG groups of 16 poses, NBUF accumulator buffers of 3 x 16 NG columns (32-column aligned)
template <int NG, int NBUF>
struct TcrShape {
    static constexpr int kPoses = 16 * NG;
    static constexpr int kThreads = NG * 128 + 64;  // + the MMA warp and the producer warp
    static constexpr uint32_t kBufCols = (3 * kPoses + 31) / 32 * 32;
    static_assert(NBUF >= 2 && NBUF * kBufCols <= kTcCols, "accumulator buffers fit the TMEM columns");
    static constexpr uint32_t kPTile = 3 * kPoses * 128;  // pose rows: 3 x kPoses rows of 128 bytes
    static constexpr size_t kSmemNeed = 1024 + 2 * kPTile + kTcrStages * kTcrRStage + 2 * 2 * 4 * kPoses * 4 +
                                        (2 * kTcrStages + 2 * NBUF + 4) * 8 + 2 * 32 + 16;
    static constexpr size_t kSmem = kSmemNeed > 116 * 1024 ? kSmemNeed : 116 * 1024;
    static_assert(3 * kPoses <= 256 && (3 * kPoses) % 16 == 0 && kPTile % 1024 == 0, "MMA shape");
};

__device__ __forceinline__ float fma_sat(float a, float b, float c) {
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Rows u, v, z of the poses lane, lane + 32, lane + 64 (< P) of pose tile
// `tile` of query d (zero rows past nh) as bf16 split-piece operand rows
// n = r P + t of the 128-byte-swizzled pose tile sP; u and v scaled by
// inv_tau and carrying 2^-100 in K lane 24.  Run by one warp; the pose
// loads of all its poses are issued before any row is written.  Kept out of
// line: inlined, its temporaries would crowd the kernel's registers.
__device__ __noinline__ void tcr_pose_rows_warp(const QueryDesc& d, int tile, int nh, int64_t slot_base,
                                                float inv_tau, int lane, int P, unsigned char* sP) {
    constexpr int J = 3;  // poses per lane (P <= 96)
    int id[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int t = lane + 32 * j, pj = tile * P + t;
        id[j] = (t < P && pj < nh) ? d.compact[pj] : -1;
    }
    PoseF ps[J];
#pragma unroll
    for (int j = 0; j < J; ++j)
        if (id[j] >= 0) ps[j] = d.slots[id[j] - slot_base];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int t = lane + 32 * j;
        if (t >= P) break;
        float c12[12];
        if (id[j] >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                c12[c] = (d.fx * ps[j].R[c] + d.cx * ps[j].R[6 + c]) * inv_tau;
                c12[4 + c] = (d.fy * ps[j].R[3 + c] + d.cy * ps[j].R[6 + c]) * inv_tau;
                c12[8 + c] = ps[j].R[6 + c];
            }
            c12[3] = (d.fx * ps[j].t[0] + d.cx * ps[j].t[2]) * inv_tau;
            c12[7] = (d.fy * ps[j].t[1] + d.cy * ps[j].t[2]) * inv_tau;
            c12[11] = ps[j].t[2];
        } else {
#pragma unroll
            for (int c = 0; c < 12; ++c) c12[c] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            uint4 ch[8];
            tc_operand_row(c12 + 4 * r, true, true, ch);
            if (r < 2) ch[3].x = kBf16Eps;  // K lane 24: 2^-100 x the records' 1
            const int n = r * P + t;
            uint4* row = reinterpret_cast<uint4*>(sP + (n >> 3) * 1024 + (n & 7) * 128);
#pragma unroll
            for (int c = 0; c < 4; ++c) row[c ^ (n & 7)] = ch[c];  // the chunks of the two K steps
        }
    }
}

// One work item of k_score_tcr, decoded by the producer warp for the others.
struct __align__(8) TcrItem {
    int64_t slot_base;  // first pose slot of the query's wave
    int32_t item;       // >= the item count: no more items
    int32_t q, tile, active, nblk, nh;
};

// PARTS: the epilogue reads a block's accumulators for its 16 poses in PARTS
// parts of 16 / PARTS poses (fewer registers of accumulator values live);
// PIPE: the next part's load is in flight while a part is computed.
// Work items flow through a two-slot queue in shared memory: the producer
// warp takes the next item from the global counter as soon as it has issued
// the record copies of the current one, decodes it, writes its pose rows
// into the slot's pose buffer and publishes it (ifull); the MMA warp and the
// epilogue warps take items from the queue in order, each at its own pace,
// and free a slot (iempty) once they have read it; the MMA warp's commit
// frees it only when the item's MMAs, which read the slot's pose rows, have
// completed.  So the next item's decoding, pose rows and first copies
// overlap the current item, and its first MMAs the current item's
// end-of-item reduction.
template <int NG, int NBUF, int PARTS, bool PIPE, bool COUNT>
__global__ void __launch_bounds__(TcrShape<NG, NBUF>::kThreads, 1) k_score_tcr(const __grid_constant__ ScoreParams p) {
    using TS = TcrShape<NG, NBUF>;
    constexpr uint32_t kTcrBufCols = TS::kBufCols;
    constexpr int P = TS::kPoses;
    constexpr int S = kTcrStages;
    constexpr int KSTEPS = 2;  // bf16 pieces: two K steps of 16
    constexpr int WMMA = 4 * NG, WPROD = WMMA + 1;
    extern __shared__ __align__(1024) unsigned char tcr_smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tcr_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sP = smem;                     // pose rows (B operand) of the two queue slots
    unsigned char* sR = sP + 2 * TS::kPTile;      // ring of record operand blocks (A operand)
    float* s_part = reinterpret_cast<float*>(sR + S * kTcrRStage);  // [2 slots][4 warp quarters][P]
    int* s_cntp = reinterpret_cast<int*>(s_part + 2 * 4 * P);        // [2][4][P]
    uint64_t* full = reinterpret_cast<uint64_t*>(s_cntp + 2 * 4 * P);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NBUF;
    uint64_t* ifull = tempty + NBUF;
    uint64_t* iempty = ifull + 2;
    TcrItem* s_info = reinterpret_cast<TcrItem*>(iempty + 2);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(s_info + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);  // the MMA's commit: the stage's MMAs have read it
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], WMMA * 32);  // every epilogue thread, once it has loaded the buffer
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&ifull[k], 1);          // the producer, once the slot's item and pose rows are written
            mbar_init(&iempty[k], WMMA + 1);  // every epilogue warp once it has read the slot, and the MMA
                                              // warp once the item's MMAs have completed
        }
        mbar_fence_init();
    }
    if (warp == WMMA) {
        tmem_alloc(tmem_slot, kTcCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int total_tiles = p.tile_prefix[p.nq];

    if (warp == WPROD) {
        // ---- producer: items into the queue, record blocks into the ring ----
        uint32_t base = 0;  // record blocks of the earlier items of this CTA (ring positions)
        for (int it = 0;; ++it) {
            const int k = it & 1;
            mbar_wait_bounded(&iempty[k], ((it >> 1) & 1u) ^ 1u, p.err);
            int item = 0;
            if (lane == 0) item = static_cast<int>(atomicAdd(p.work_counter, 1u));
            item = __shfl_sync(0xffffffffu, item, 0);
            TcrItem I;
            I.item = item;
            I.q = I.tile = I.active = I.nblk = I.nh = 0;
            I.slot_base = 0;
            if (item < total_tiles) {
                int lo = 0, hi = p.nq - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (p.tile_prefix[mid] <= item) lo = mid;
                    else hi = mid - 1;
                }
                I.q = lo;
                I.tile = item - p.tile_prefix[lo];
                I.active = I.tile < p.ntiles[lo] ? 1 : 0;
                const int m = I.active ? p.qs[lo].m : 0;
                I.nblk = (m + kTcrRecs - 1) / kTcrRecs;
                I.nh = p.n_hyp[lo];
                I.slot_base = 4 * p.wq[lo].s_begin;
            }
            if (I.active) {
                const QueryDesc& d = p.qd[I.q];
                tcr_pose_rows_warp(d, I.tile, I.nh, I.slot_base, 1.0f / sqrtf(d.tau2), lane, P, sP + k * TS::kPTile);
                // the generic-proxy writes become visible to the tensor core's reads
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            if (lane == 0) s_info[k] = I;
            __syncwarp();
            if (lane == 0) mbar_arrive(&ifull[k]);
            if (item >= total_tiles) break;
            if (I.active) {
                const QueryDesc& d = p.qd[I.q];
                for (int b = 0; b < I.nblk; ++b) {
                    const uint32_t gb = base + b;
                    const uint32_t st = gb % S;
                    mbar_wait_bounded(&empty[st], ((gb / S) & 1u) ^ 1u, p.err);
                    if (lane == 0) {
                        mbar_arrive_expect_tx(&full[st], kTcrRStage);
                        bulk_g2s(sR + st * kTcrRStage, d.tc_rec + static_cast<int64_t>(b) * kTcrRecs * 8, kTcrRStage,
                                 &full[st]);
                    }
                    __syncwarp();
                }
            }
            base += static_cast<uint32_t>(I.nblk);
        }
    } else if (warp == WMMA) {
        // ---- MMA warp: the whole warp walks the blocks (it stays converged); one elected lane issues ----
        constexpr uint32_t idesc = umma_idesc_bf16(kTcrRecs, 3 * P);
        const uint64_t rdesc = umma_desc_k_sw128(smem_u32(sR));
        uint32_t base = 0;
        int it = 0;
        for (;; ++it) {
            const int k = it & 1;
            mbar_wait_bounded(&ifull[k], (it >> 1) & 1u, p.err);
            const TcrItem I = s_info[k];
            if (I.item >= total_tiles) break;
            const uint64_t pdesc = umma_desc_k_sw128(smem_u32(sP + k * TS::kPTile));
            for (int b = 0; b < I.nblk; ++b) {
                const uint32_t gb = base + b;
                const uint32_t st = gb % S, buf = gb % NBUF;
                mbar_wait_bounded(&tempty[buf], ((gb / NBUF) & 1u) ^ 1u, p.err);
                mbar_wait_bounded(&full[st], (gb / S) & 1u, p.err);
                tc_fence_after();
                const uint64_t ad0 = rdesc + ((st * kTcrRStage) >> 4);
                const uint32_t d0 = tmem_base + buf * kTcrBufCols;
                if (elect_one()) {
#pragma unroll
                    for (int kk = 0; kk < KSTEPS; ++kk)
                        umma_bf16(d0, ad0 + ((kk * 32) >> 4), pdesc + ((kk * 32) >> 4), idesc, kk > 0 ? 1u : 0u);
                    umma_commit(&tfull[buf]);
                    umma_commit(&empty[st]);
                }
                __syncwarp();
            }
            // the slot is free once every MMA issued so far (those that read its pose rows) has completed
            if (elect_one()) {
                if (I.nblk > 0) umma_commit(&iempty[k]);
                else mbar_arrive(&iempty[k]);
            }
            __syncwarp();
            base += static_cast<uint32_t>(I.nblk);
        }
        // the last items' commits have landed before the CTA (and its barriers) can go
        for (int l = it - 2 > 0 ? it - 2 : 0; l < it; ++l) mbar_wait_bounded(&iempty[l & 1], (l >> 1) & 1u, p.err);
    } else if (warp < WMMA) {
        // ---- epilogue warps ----
        const int g = warp >> 2, wq = warp & 3;
        const uint32_t lane_addr = tmem_base + (static_cast<uint32_t>(wq * 32) << 16) + 16 * g;
        uint32_t base = 0;
        for (int it = 0;; ++it) {
            const int k = it & 1;
            mbar_wait_bounded(&ifull[k], (it >> 1) & 1u, p.err);
            const TcrItem I = s_info[k];
            __syncwarp();
            if (lane == 0) mbar_arrive(&iempty[k]);
            if (I.item >= total_tiles) break;
            if (!I.active) continue;
            const QueryDesc& d = p.qd[I.q];
            const int nblk = I.nblk;
            // running sums of this lane's records for poses 16 g .. 16 g + 15 (pairs of poses)
            uint64_t acc2[8];
            uint32_t cnt2[8];  // with COUNT: inliers of poses 2i (low 16 bits) and 2i + 1 (high 16 bits)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc2[i] = f2_pack(0.f, 0.f);
                cnt2[i] = 0u;
            }
            // this thread's record of every block: {-x / tau, -y / tau, w tau^2, 0}
            const float* te = reinterpret_cast<const float*>(d.tc_e + wq * 32 + lane);
            float ex = __ldg(te), ey = __ldg(te + 1), ew = __ldg(te + 2);  // block 0
            // one block: accumulator buffer BUF (a compile-time constant, so that its
            // TMEM addresses and barrier are loop-invariant)
            auto do_block = [&](auto buf_c, int b) {
                constexpr uint32_t buf = decltype(buf_c)::value;
                const uint32_t gb = base + b;
                // the next block's pixel and weight, in flight during this block
                const float* tn = te + static_cast<int64_t>(b + 1 < nblk ? b + 1 : b) * (kTcrRecs * 4);
                const float ex_n = __ldg(tn), ey_n = __ldg(tn + 1), ew_n = __ldg(tn + 2);
                mbar_wait_bounded(&tfull[buf], (gb / NBUF) & 1u, p.err);
                tc_fence_after();
                const uint32_t ta = lane_addr + buf * kTcrBufCols;
                const uint64_t nx2 = f2_pack(ex, ex), ny2 = f2_pack(ey, ey), w2 = f2_pack(ew, ew);
                constexpr int H = PARTS, KH = 8 / H, W = 16 / H;  // parts, pose pairs and columns per part
                uint32_t z[PIPE ? 2 : 1][3][W];                      // u, v, z columns of a part (two sets: PIPE)
                auto load_part = [&](int h, uint32_t (&zs)[3][W]) {
                    tmem_ld_nowait<W>(ta + W * h, zs[0]);
                    tmem_ld_nowait<W>(ta + P + W * h, zs[1]);
                    tmem_ld_nowait<W>(ta + 2 * P + W * h, zs[2]);
                };
                auto ready = [&](uint32_t (&zs)[3][W]) {
                    tmem_regs_ready<W>(zs[0]);
                    tmem_regs_ready<W>(zs[1]);
                    tmem_regs_ready<W>(zs[2]);
                };
                if constexpr (PIPE) {
                    load_part(0, z[0]);
                    tmem_wait_ld();
                    ready(z[0]);
                }
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    uint32_t (&zc)[3][W] = z[PIPE ? (h & 1) : 0];
                    if constexpr (PIPE) {
                        if (h + 1 < H) load_part(h + 1, z[(h + 1) & 1]);
                    } else {
                        load_part(h, zc);
                        tmem_wait_ld();
                        ready(zc);
                    }
                    if (h == H - 1) {
                        // every load of this buffer has completed
                        tc_fence_before();
                        mbar_arrive(&tempty[buf]);
                    }
#pragma unroll
                    for (int kh = 0; kh < KH; ++kh) {
                        const int k = h * KH + kh;  // pose pair of the group's 16
                        const float z0 = __uint_as_float(zc[2][2 * kh]), z1 = __uint_as_float(zc[2][2 * kh + 1]);
                        const float i0 = rcp_approx(fmaxf(z0, 0.0f)), i1 = rcp_approx(fmaxf(z1, 0.0f));
                        const uint64_t iz2 = f2_pack(i0, i1);
                        const uint64_t du2 = f2_fma(
                            f2_pack(__uint_as_float(zc[0][2 * kh]), __uint_as_float(zc[0][2 * kh + 1])), iz2, nx2);
                        const uint64_t dv2 = f2_fma(
                            f2_pack(__uint_as_float(zc[1][2 * kh]), __uint_as_float(zc[1][2 * kh + 1])), iz2, ny2);
                        float du0, du1, q0, q1;
                        f2_unpack(du2, du0, du1);
                        f2_unpack(f2_mul(dv2, dv2), q0, q1);
                        if (COUNT) {
                            // the unclamped scaled residual decides the inlier count (NaN: not an inlier)
                            const float r0 = fmaf(du0, du0, q0), r1 = fmaf(du1, du1, q1);
                            cnt2[k] += ((r0 < 1.0f) ? 1u : 0u) + ((r1 < 1.0f) ? 0x10000u : 0u);
                            acc2[k] = f2_fma(w2, f2_pack(fminf(r0, 1.0f), fminf(r1, 1.0f)), acc2[k]);
                        } else {
                            acc2[k] = f2_fma(w2, f2_pack(fma_sat(du0, du0, q0), fma_sat(du1, du1, q1)), acc2[k]);
                        }
                    }
                    if constexpr (PIPE) {
                        if (h + 1 < H) {
                            tmem_wait_ld();
                            ready(z[(h + 1) & 1]);
                        }
                    }
                }
                ex = ex_n;
                ey = ey_n;
                ew = ew_n;
            };
            // blocks alternate between the two buffers in the CTA's block order (gb);
            // the item's first block takes buffer base mod 2
            using B0 = std::integral_constant<uint32_t, 0>;
            using B1 = std::integral_constant<uint32_t, 1>;
            static_assert(NBUF == 2, "the block loop is unrolled over two accumulator buffers");
            int b = 0;
            if ((base & 1u) == 0u) {
                for (; b + 1 < nblk; b += 2) {
                    do_block(B0{}, b);
                    do_block(B1{}, b + 1);
                }
                if (b < nblk) do_block(B0{}, b);
            } else {
                for (; b + 1 < nblk; b += 2) {
                    do_block(B1{}, b);
                    do_block(B0{}, b + 1);
                }
                if (b < nblk) do_block(B1{}, b);
            }
            // sums over the warp's 32 records per pose: halving exchanges leave pose
            // (lane >> 1) of the group's 16 in lanes 2 (lane >> 1) and 2 (lane >> 1) + 1
            float v[16];
            int c[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                f2_unpack(acc2[i], v[2 * i], v[2 * i + 1]);
                c[2 * i] = static_cast<int>(cnt2[i] & 0xffffu);
                c[2 * i + 1] = static_cast<int>(cnt2[i] >> 16);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int off = 16 >> s, half = 8 >> s;
                const bool upper = (lane & off) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const float send = upper ? v[i] : v[half + i];
                    const float keep = upper ? v[half + i] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                    if (COUNT) {
                        const int cs = upper ? c[i] : c[half + i];
                        const int ck = upper ? c[half + i] : c[i];
                        c[i] = ck + __shfl_xor_sync(0xffffffffu, cs, off);
                    }
                }
            }
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            if (COUNT) c[0] += __shfl_xor_sync(0xffffffffu, c[0], 1);
            if ((lane & 1) == 0) {
                s_part[(k * 4 + wq) * P + 16 * g + (lane >> 1)] = v[0];
                if (COUNT) s_cntp[(k * 4 + wq) * P + 16 * g + (lane >> 1)] = c[0];
            }
            asm volatile("bar.sync 1, %0;" ::"n"(WMMA * 32) : "memory");
            if (warp < (P + 31) / 32) {
                const int e = tid;  // pose of the tile
                const int j = I.tile * P + e;
                const bool valid = e < P && j < I.nh;
                uint32_t id = 0xffffffffu, rd = 0xffffffffu, sb = 0xffffffffu;
                if (valid) {
                    // the four warp quarters (records 0-31, 32-63, ... of every block) in order
                    const float* sp = s_part + k * 4 * P;
                    const float sc = ((sp[e] + sp[P + e]) + sp[2 * P + e]) + sp[3 * P + e];
                    const int ct =
                        COUNT ? s_cntp[k * 4 * P + e] + s_cntp[(k * 4 + 1) * P + e] + s_cntp[(k * 4 + 2) * P + e] +
                                    s_cntp[(k * 4 + 3) * P + e]
                                  : 0;
                    id = static_cast<uint32_t>(d.compact[j]);
                    rd = static_cast<uint32_t>((id >> 2) / static_cast<uint32_t>(d.batch));
                    sb = __float_as_uint(sc);
                    if (d.score_by_id) d.score_by_id[id - I.slot_base] = sc;
                    if (COUNT && d.count_by_id) d.count_by_id[id - I.slot_base] = ct;
                }
                // per round, the minimum (score bits, pose id) of the warp, then one atomic
                unsigned long long kv = valid ? ((static_cast<unsigned long long>(sb) << 32) | id) : ~0ull;
                bool pending = valid;
                while (__any_sync(0xffffffffu, pending)) {
                    const int first = __ffs(__ballot_sync(0xffffffffu, pending)) - 1;
                    const uint32_t r0 = __shfl_sync(0xffffffffu, rd, first);
                    unsigned long long v2 = (pending && rd == r0) ? kv : ~0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v2, o);
                        v2 = u < v2 ? u : v2;
                    }
                    if (lane == first) atomicMin(reinterpret_cast<unsigned long long*>(&d.round_best[r0]), v2);
                    if (rd == r0) pending = false;
                }
            }
            base += static_cast<uint32_t>(nblk);
        }
    }
    // every MMA completed before the epilogue read its accumulator
    tc_fence_before();
    __syncthreads();
    if (warp == WMMA) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTcCols);
    }
}

// tensor-core scoring variants: records per MMA x epilogue groups x bf16 or TF32 pieces
struct TcVariant {
    int nb, ng;
    bool bf;
    int threads;
    size_t smem;
    void (*fn)(ScoreParams);
    void (*fn_count)(ScoreParams);
    int poses;  // poses per work item
    int mode;   // QueryDesc::tc_mode of the operand rows it reads
};
#define IMLOC_TC_VARIANT(NB, NG, BF)                                                              \
    {NB, NG, BF, TcShape<NB, NG>::kThreads, TcShape<NB, NG>::kSmem, k_score_tc<NB, NG, BF, false>, \
     k_score_tc<NB, NG, BF, true>, kTcPoses, BF ? 1 : 0}
#define IMLOC_TCR_VARIANT(NG, NBUF, PARTS, PIPE)                                                         \
    {kTcrRecs, NG, true, TcrShape<NG, NBUF>::kThreads, TcrShape<NG, NBUF>::kSmem,                          \
     k_score_tcr<NG, NBUF, PARTS, PIPE, false>, k_score_tcr<NG, NBUF, PARTS, PIPE, true>, TcrShape<NG, NBUF>::kPoses, 2}
static const TcVariant kTcVariants[] = {
    // records on the M side (128-record blocks x 16 NG-pose items, bf16 pieces, 2 accumulator buffers)
    IMLOC_TCR_VARIANT(5, 2, 2, false),  // 0: 80-pose items, accumulators read in halves
    IMLOC_TCR_VARIANT(5, 2, 4, true),   // 1: 80-pose items, read in quarters, the next quarter in flight
    IMLOC_TCR_VARIANT(4, 2, 1, false),  // 2: 64-pose items, read whole (16 columns per row)
    // poses on the M side (128-pose tiles)
    IMLOC_TC_VARIANT(80, 5, true),      // 3: 80-record blocks (2 TMEM buffers), 5 groups x 16 records, bf16 pieces
    IMLOC_TC_VARIANT(80, 5, false),     // 4: as 3 with TF32 pieces (3 K steps)
};
#undef IMLOC_TC_VARIANT
#undef IMLOC_TCR_VARIANT
constexpr int kNumTcVariants = sizeof(kTcVariants) / sizeof(kTcVariants[0]);

// score kernel variants the autotuner chooses from (same results, different speed)
struct ScoreVariant {
    int threads, ht;
    void (*fn)(ScoreParams);
    void (*fn_count)(ScoreParams);
    void (*fused)(ScoreParams);
    void (*fused_count)(ScoreParams);
};
// MF: occupancy bound of the fused instance = the CTAs per SM of the unfused one,
// so that the replay code does not cost the scoring loop any occupancy
#define IMLOC_SCORE_VARIANT(T, H, M, U, MF)                                                            \
    {T, H, k_score<T, H, false, M, U, false, MF>, k_score<T, H, true, M, U, false, MF>,                 \
     k_score<T, H, false, M, U, true, MF>, k_score<T, H, true, M, U, true, MF>}
static const ScoreVariant kScoreVariants[] = {
    IMLOC_SCORE_VARIANT(128, 4, 1, 1, 3),  // 512-pose tiles; ~144 registers: 3 CTAs / SM
    IMLOC_SCORE_VARIANT(128, 4, 4, 1, 4),  // <= 128 registers: 4 CTAs / SM
    IMLOC_SCORE_VARIANT(128, 4, 3, 2, 3),
    IMLOC_SCORE_VARIANT(256, 2, 2, 2, 2),
    IMLOC_SCORE_VARIANT(256, 2, 3, 1, 3),  // <= 85 registers: 3 CTAs / SM
    IMLOC_SCORE_VARIANT(128, 2, 5, 1, 5),  // 256-pose tiles (finer work items): 5 CTAs / SM
    IMLOC_SCORE_VARIANT(128, 2, 6, 2, 5),  // <= 85 registers: 6 CTAs / SM
    IMLOC_SCORE_VARIANT(64, 4, 6, 1, 5),   // 256-pose tiles, 2 warps per CTA
};
#undef IMLOC_SCORE_VARIANT
constexpr int kNumScoreVariants = sizeof(kScoreVariants) / sizeof(kScoreVariants[0]);

static size_t score_smem_bytes(bool count, int tile) {
    return sizeof(ScorePair) * kWinPairs + sizeof(float) * tile + (count ? sizeof(int) * tile : 0);
}

// ============================================================================
// host orchestration
// ============================================================================
struct HostQuery {
    const float *x, *y, *X, *Y, *Z, *w;
    const int64_t* d_off;
    int32_t q_off;
    const int32_t* d_count;
    int64_t n_host;
    int64_t n_cap;
    uint8_t* mask;
    int32_t* fixidx_base; // fixed-set indices at the same offsets as the correspondences (null: allocate)
    imloc_result* d_result;
    imloc_camera cam;
    imloc_ransac_opts o;
    // tests
    const PoseF* inject;
    int64_t n_inject;
    float* score_by_id;
    int32_t* count_by_id;
    int32_t* triples;
    PoseF* slots_out;
    uint64_t* round_best_out;
    uint64_t* rescored_out;
};


template <typename K, typename P>
static int launch_cluster(K kernel, const P& params, int grid, int block, size_t smem, int cluster, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    IMLOC_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, params));
    return IMLOC_OK;
}

// Dynamic shared memory beyond the 48 KB default needs the function's opt-in.
template <typename K>
static int allow_smem(K kernel, size_t smem) {
    static std::mutex mu;
    static std::map<const void*, size_t> done;  // largest size already allowed per kernel
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(reinterpret_cast<const void*>(kernel));
    if (it != done.end() && it->second >= smem) return IMLOC_OK;
    IMLOC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    done[reinterpret_cast<const void*>(kernel)] = smem;
    return IMLOC_OK;
}

template <typename K>
static int max_clusters(K kernel, int block, size_t smem, int cluster, int* out) {
    if (smem > 0) {
        const int rc = allow_smem(kernel, smem);
        if (rc != IMLOC_OK) return rc;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * 64);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    IMLOC_CUDA_TRY(cudaOccupancyMaxActiveClusters(out, kernel, &cfg));
    return IMLOC_OK;
}

// CTAs per query in the replay: the largest cluster (8 down to 1 CTAs, at
// most IMLOC_REPLAY_CLUSTER when set) of which all nq can be resident at once
// (a query whose cluster waits for another to finish adds a whole replay to
// the kernel time).  With one CTA per SM, 16 clusters of 8 do not fit the GPCs
// of a 152-SM GB300 (15 do), 23 of 6 do.
template <typename ACC>
static int replay_cluster_size(imloc_ctx* ctx, int nq, int* cl_out) {
    static const int kCl[kReplayClusterChoices] = {8, 7, 6, 5, 4, 3, 2, 1};
    // IMLOC_REPLAY_CLUSTER=<k>: at most k CTAs per query
    static const int cap = [] {
        const char* env = getenv("IMLOC_REPLAY_CLUSTER");
        return env ? std::min(std::max(atoi(env), 1), 8) : 8;
    }();
    const int a = sizeof(ACC) == 8 ? 1 : 0;
    for (int i = 0; i < kReplayClusterChoices; ++i) {
        if (kCl[i] > cap) continue;
        int& occ = ctx->replay_occ[a][i];
        if (occ == 0) {
            int v = 0;
            const int rc = max_clusters(k_replay<ACC>, replay_threads<ACC>(), kReplayStageBytes, kCl[i], &v);
            if (rc != IMLOC_OK) return rc;
            occ = v > 0 ? v : -1;
        }
        if (occ >= nq) {
            *cl_out = kCl[i];
            if (getenv("IMLOC_VERBOSE"))
                fprintf(stderr, "imloc: replay of %d queries in clusters of %d (%d co-resident)\n", nq, kCl[i], occ);
            return IMLOC_OK;
        }
    }
    *cl_out = 1;
    return IMLOC_OK;
}

static int64_t comb3(int64_t m) { return m < 3 ? 0 : m * (m - 1) * (m - 2) / 6; }

static int launch_tiles(imloc_ctx* ctx, const StepBuffers& b, int nq, int tile, cudaStream_t stream) {
    TilesParams tp{b.d_qs, b.d_nhyp, b.d_tiles, b.d_tiles + nq + 1, b.d_tiles + 2 * nq + 1, b.d_counter, nq, tile};
    ProfScope prof(ctx, stream, "k_tiles");
    k_tiles<<<1, 1024, 0, stream>>>(tp);
    IMLOC_CUDA_TRY(cudaGetLastError());
    prof.end();
    return IMLOC_OK;
}

// Upper bound of the work items of a wave with tiles of `tile` poses.
static int64_t max_items_of(int64_t total_samples, int nq, int tile) {
    return std::max<int64_t>(1, (total_samples * 4 + tile - 1) / tile + nq);
}

// Autotuner of the score kernel: every variant computes bitwise-identical
// scores (same record order and summation structure per pose), so the
// variants are timed on the live wave (the kernel is idempotent: it rewrites
// the same scores and re-applies the same atomic minima; the tile table is
// rebuilt for each variant's tile size) and the fastest is kept for the
// context.  IMLOC_SCORE_VARIANT=<k> forces variant k.
static int tune_score(imloc_ctx* ctx, const StepBuffers& b, int nq, const ScoreParams& scp, bool counts,
                      int64_t total_samples, cudaStream_t stream) {
    if (const char* env = getenv("IMLOC_SCORE_VARIANT")) {
        const int k = atoi(env);
        ctx->score_variant = (k >= 0 && k < kNumScoreVariants) ? k : 0;
        return IMLOC_OK;
    }
    cudaEvent_t e0, e1;
    IMLOC_CUDA_TRY(cudaEventCreate(&e0));
    IMLOC_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best = 0;
    for (int rep = 0; rep < 2; ++rep)
        for (int v = 0; v < kNumScoreVariants; ++v) {
            const ScoreVariant& V = kScoreVariants[v];
            const int tile = V.threads * V.ht;
            const size_t smem = score_smem_bytes(counts, tile);
            auto kern = counts ? V.fn_count : V.fn;
            int n_clusters = 0;
            int rc = max_clusters(kern, V.threads, smem, kScoreCluster, &n_clusters);
            if (rc != IMLOC_OK || n_clusters <= 0) continue;
            const int grid = static_cast<int>(std::min<int64_t>(n_clusters, max_items_of(total_samples, nq, tile)));
            rc = launch_tiles(ctx, b, nq, tile, stream);
            if (rc != IMLOC_OK) return rc;
            IMLOC_CUDA_TRY(cudaEventRecord(e0, stream));
            rc = launch_cluster(kern, scp, grid * kScoreCluster, V.threads, smem, kScoreCluster, stream);
            if (rc != IMLOC_OK) return rc;
            IMLOC_CUDA_TRY(cudaEventRecord(e1, stream));
            IMLOC_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            IMLOC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms < best_ms) { best_ms = ms; best = v; }
            if (rep == 1 && getenv("IMLOC_VERBOSE"))
                fprintf(stderr, "imloc: score variant %d (%d threads x %d poses) %.3f ms\n", v, V.threads, V.ht, ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->score_variant = best;
    ctx->score_variant_ms = best_ms;
    return IMLOC_OK;
}

// IMLOC_FUSE=1 / IMLOC_NO_FUSE=1 force the fused / unfused form
static bool fuse_of(bool dflt) { return getenv("IMLOC_NO_FUSE") ? false : (getenv("IMLOC_FUSE") ? true : dflt); }

// Which scoring kernel an unfused call takes: the tensor-core one when the
// call has enough pose tiles (~1.2 poses per minimal set, 128 per tile) for
// two per SM, the FP32 one otherwise (a single query: the cluster-split FP32
// kernel spreads it over more SMs).  imloc_set_scoring, else IMLOC_SCORE_TC=0
// / 1, forces either.
static bool score_tc_enabled(const imloc_ctx* ctx, int64_t total_samples) {
    if (ctx->scoring_kernel >= 0) return ctx->scoring_kernel == 1;
    const char* env = getenv("IMLOC_SCORE_TC");
    if (env) return atoi(env) != 0;
    return total_samples * 6 / 5 >= 2LL * std::max(1, ctx->sm_count) * kTcPoses;
}

// The tensor-core scoring variant: imloc_set_scoring's, else IMLOC_TC_VARIANT=<k>, else 0
static int tc_variant(const imloc_ctx* ctx) {
    if (ctx->scoring_tc_variant >= 0) return std::min(ctx->scoring_tc_variant, kNumTcVariants - 1);
    const char* env = getenv("IMLOC_TC_VARIANT");
    return env ? std::min(std::max(atoi(env), 0), kNumTcVariants - 1) : 0;
}

int run_step(imloc_ctx* ctx, const StepBuffers& b, int nq, int n_init, int64_t total_samples, bool want_counts,
             cudaStream_t stream) {
    int rc;
    if (n_init > 0) {
        SetupParams sp{b.d_qd, b.d_qs, b.d_nhyp_all, b.nhyp_all_len, b.d_init};
        ProfScope prof(ctx, stream, "k_setup");
        k_setup<<<n_init * kSetupBlocks, 256, 0, stream>>>(sp);
        IMLOC_CUDA_TRY(cudaGetLastError());
        prof.end();
        if (b.bf16) {
            ProfScope prof2(ctx, stream, "k_setup_bf16");
            k_setup_bf16<<<n_init, 512, 0, stream>>>(b.d_qd, b.d_qs, b.d_init);
            IMLOC_CUDA_TRY(cudaGetLastError());
            prof2.end();
        }
    }
    if (total_samples > 0) {
        SampleParams sp{b.d_qd, b.d_qs, b.d_wq, b.d_prefix, b.d_nhyp, total_samples, nq};
        const int64_t blocks = (total_samples + 127) / 128;
        ProfScope prof(ctx, stream, "k_sample_p3p");
        k_sample_p3p<<<static_cast<unsigned>(blocks), 128, 0, stream>>>(sp);
        IMLOC_CUDA_TRY(cudaGetLastError());
        prof.end();
    }
    ScoreParams scp{b.d_qd,       b.d_qs,      b.d_wq, b.d_nhyp,   b.d_tiles, b.d_tiles + nq + 1, b.d_tiles + 2 * nq + 1,
                    b.d_counter, nq,          ctx->d_err, b.d_rescored};
    // the fused kernel scores and replays each query when its last item is done
    // (replays overlap the scoring of later queries: worth it with many
    // queries); otherwise the scoring runs alone, followed by the replay kernel.
    const bool fuse = fuse_of(b.fuse) && !b.bf16;
    if (b.bf16) {
        // bf16-packed records with FP32 rescoring: the FP32 kernel's work queue and cluster split
        rc = launch_tiles(ctx, b, nq, kBfTile, stream);
        if (rc != IMLOC_OK) return rc;
        auto kern = want_counts ? k_score_bf16<true> : k_score_bf16<false>;
        const size_t smem = score_bf16_smem_bytes();
        int n_clusters = 0;
        rc = max_clusters(kern, kBfThreads, smem, kScoreCluster, &n_clusters);
        if (rc != IMLOC_OK) return rc;
        const int grid_clusters =
            static_cast<int>(std::min<int64_t>(std::max(1, n_clusters), max_items_of(total_samples, nq, kBfTile)));
        ProfScope prof(ctx, stream, "k_score_bf16");
        rc = launch_cluster(kern, scp, grid_clusters * kScoreCluster, kBfThreads, smem, kScoreCluster, stream);
        if (rc != IMLOC_OK) return rc;
        prof.end();
    } else if (b.tc && !fuse) {
        // projections on the tensor cores: one persistent CTA per SM
        const TcVariant& TV = kTcVariants[tc_variant(ctx)];
        rc = launch_tiles(ctx, b, nq, TV.poses, stream);
        if (rc != IMLOC_OK) return rc;
        auto kern = want_counts ? TV.fn_count : TV.fn;
        IMLOC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(TV.smem)));
        const int grid = static_cast<int>(
            std::min<int64_t>(std::max(1, ctx->sm_count), max_items_of(total_samples, nq, TV.poses)));
        ProfScope prof(ctx, stream, "k_score_tc");
        kern<<<grid, TV.threads, TV.smem, stream>>>(scp);
        IMLOC_CUDA_TRY(cudaGetLastError());
        prof.end();
    } else {
        // autotune the score kernel variant once per context on a large enough wave
        if (ctx->score_variant < 0 &&
            (max_items_of(total_samples, nq, kMaxTileHyps) >= 64 || getenv("IMLOC_SCORE_VARIANT"))) {
            rc = tune_score(ctx, b, nq, scp, want_counts, total_samples, stream);
            if (rc != IMLOC_OK) return rc;
        }
        const ScoreVariant& V = kScoreVariants[ctx->score_variant >= 0 ? ctx->score_variant : 0];
        const int tile = V.threads * V.ht;
        const size_t score_smem = score_smem_bytes(want_counts, tile);
        const int64_t max_items = max_items_of(total_samples, nq, tile);
        rc = launch_tiles(ctx, b, nq, tile, stream);
        if (rc != IMLOC_OK) return rc;
        auto score_kernel = fuse ? (want_counts ? V.fused_count : V.fused) : (want_counts ? V.fn_count : V.fn);
        int n_clusters = 0;
        rc = max_clusters(score_kernel, V.threads, score_smem, kScoreCluster, &n_clusters);
        if (rc != IMLOC_OK) return rc;
        const int grid_clusters = static_cast<int>(std::min<int64_t>(std::max(1, n_clusters), max_items));
        ProfScope prof(ctx, stream, "k_score");
        rc = launch_cluster(score_kernel, scp, grid_clusters * kScoreCluster, V.threads, score_smem, kScoreCluster,
                            stream);
        if (rc != IMLOC_OK) return rc;
        prof.end();
    }
    {
        ReplayParams rp{b.d_qd, b.d_qs, b.d_wq, ctx->d_err};
        // queries with FP64 accumulation replay in their own kernel after the scoring
        if (!fuse || b.any_fp64) {
            ProfScope prof(ctx, stream, "k_replay");
            if (!fuse) {
                int cl = 1;
                rc = replay_cluster_size<float>(ctx, nq, &cl);
                if (rc != IMLOC_OK) return rc;
                rc = launch_cluster(k_replay<float>, rp, nq * cl, replay_threads<float>(), kReplayStageBytes, cl, stream);
                if (rc != IMLOC_OK) return rc;
            }
            if (b.any_fp64) {
                int cl = 1;
                rc = replay_cluster_size<double>(ctx, nq, &cl);
                if (rc != IMLOC_OK) return rc;
                rc = launch_cluster(k_replay<double>, rp, nq * cl, replay_threads<double>(), kReplayStageBytes, cl, stream);
                if (rc != IMLOC_OK) return rc;
            }
            prof.end();
        }
    }
    return IMLOC_OK;
}

int ransac_impl(imloc_ctx* ctx, int nq, const HostQuery* hq, cudaStream_t stream, bool want_counts) {
    if (nq <= 0) return IMLOC_ERR_INVALID_ARG;
    // ---- per-query host-known sizes and the wave schedule ----
    std::vector<int64_t> H(nq), B(nq), R(nq);
    int64_t R_max = 0;
    bool adaptive = false;
    for (int q = 0; q < nq; ++q) {
        const imloc_ransac_opts& o = hq[q].o;
        if (!(o.tau_px > 0.0) || o.max_score_corr < 3 || o.batch <= 0 || o.max_iters <= 0 || o.lo_iters < 0 ||
            o.final_iters < 0 || !(hq[q].cam.fx != 0.0f) || !(hq[q].cam.fy != 0.0f))
            return IMLOC_ERR_INVALID_ARG;
        if (!hq[q].x || !hq[q].y || !hq[q].X || !hq[q].Y || !hq[q].Z || !hq[q].w) return IMLOC_ERR_INVALID_ARG;
        if (hq[q].inject) {
            H[q] = hq[q].n_inject;
            B[q] = std::min<int64_t>(o.batch, std::max<int64_t>(1, H[q]));
        } else if (o.enumerate_all) {
            if (hq[q].d_off || hq[q].d_count) return IMLOC_ERR_INVALID_ARG;  // needs a host-known N
            const int64_t m = std::min<int64_t>(hq[q].n_host, o.max_score_corr);
            H[q] = comb3(m);
            if (H[q] > (int64_t(1) << 24)) return IMLOC_ERR_INVALID_ARG;
            B[q] = std::max<int64_t>(1, H[q]);
        } else {
            H[q] = o.max_iters;
            B[q] = o.batch;
        }
        if (H[q] <= 0) H[q] = 0;
        R[q] = H[q] > 0 ? (H[q] + B[q] - 1) / B[q] : 0;
        R_max = std::max(R_max, R[q]);
        if (o.p_miss > 0.0 && !o.enumerate_all && !hq[q].inject) adaptive = true;
    }
    std::vector<std::pair<int64_t, int64_t>> waves;
    if (!adaptive) {
        waves.push_back({0, std::max<int64_t>(R_max, 1)});
    } else {
        int64_t r = 0, len = 1;
        while (r < R_max) {
            const int64_t e = std::min(R_max, r + len);
            waves.push_back({r, e});
            r = e;
            if (waves.size() >= 2) len *= 2;
        }
        if (waves.empty()) waves.push_back({0, 1});
    }
    const int W = static_cast<int>(waves.size());
    if ((hq[0].score_by_id || hq[0].count_by_id || hq[0].triples || hq[0].slots_out) && W != 1)
        return IMLOC_ERR_INVALID_ARG;
    std::vector<WaveQ> wq(static_cast<size_t>(W) * nq);
    std::vector<int64_t> wprefix(static_cast<size_t>(W) * (nq + 1));
    std::vector<int64_t> wtotal(W, 0);
    std::vector<int64_t> max_wave_samples(nq, 0);
    for (int w = 0; w < W; ++w) {
        int64_t acc = 0;
        for (int q = 0; q < nq; ++q) {
            const int64_t sb = std::min(waves[w].first * B[q], H[q]);
            const int64_t se = std::min(waves[w].second * B[q], H[q]);
            WaveQ& x = wq[static_cast<size_t>(w) * nq + q];
            x.s_begin = sb;
            x.n_samples = static_cast<int32_t>(se - sb);
            x.r0 = static_cast<int32_t>(waves[w].first);
            x.r1 = static_cast<int32_t>(waves[w].second);
            x.pad = 0;
            wprefix[static_cast<size_t>(w) * (nq + 1) + q] = acc;
            acc += se - sb;
            max_wave_samples[q] = std::max(max_wave_samples[q], se - sb);
        }
        wprefix[static_cast<size_t>(w) * (nq + 1) + nq] = acc;
        wtotal[w] = acc;
    }

    // ---- workspace ----
    // Scoring form: the tensor-core kernel (unfused) when the call is large
    // enough for it; else the FP32 kernel, fused with the replay for >= 32
    // queries.  On 256 queries the tensor-core kernel plus a replay kernel
    // beats the fused FP32 form (15.0 vs 16.2 ms).
    int64_t all_samples = 0;
    for (int q = 0; q < nq; ++q) all_samples += H[q];
    // bf16-packed scoring when every query of the call asks for it
    bool bf16_on = true;
    for (int q = 0; q < nq; ++q) bf16_on = bf16_on && hq[q].o.score_bf16 != 0;
    const bool want_tc = score_tc_enabled(ctx, all_samples) && !bf16_on;
    const bool dflt_fuse = nq >= 32 && !want_tc && !bf16_on;
    bool tc_on = want_tc && !fuse_of(dflt_fuse);
    std::vector<QueryDesc> qd(nq);
    int64_t est_hyp = 0;
    for (int q = 0; q < nq; ++q) {
        const HostQuery& h = hq[q];
        const imloc_ransac_opts& o = h.o;
        QueryDesc& d = qd[q];
        memset(&d, 0, sizeof(d));
        d.x = h.x; d.y = h.y; d.X = h.X; d.Y = h.Y; d.Z = h.Z; d.w = h.w;
        d.d_off = h.d_off; d.q_off = h.q_off; d.d_count = h.d_count; d.n_host = h.n_host;
        d.mask = h.mask;
        d.result = h.d_result;
        d.fx = h.cam.fx; d.fy = h.cam.fy; d.cx = h.cam.cx; d.cy = h.cam.cy;
        {
            const double ifx = 1.0 / static_cast<double>(h.cam.fx), ify = 1.0 / static_cast<double>(h.cam.fy);
            d.ifx_hi = static_cast<float>(ifx);
            d.ifx_lo = static_cast<float>(ifx - static_cast<double>(d.ifx_hi));
            d.ify_hi = static_cast<float>(ify);
            d.ify_lo = static_cast<float>(ify - static_cast<double>(d.ify_hi));
        }
        d.tau2 = static_cast<float>(o.tau_px * o.tau_px);
        const double cs = o.cauchy_scale > 0.0 ? o.cauchy_scale : o.tau_px;
        d.cauchy2 = static_cast<float>(cs * cs);
        d.m_cap = o.max_score_corr;
        d.batch = static_cast<int32_t>(B[q]);
        d.hyps = static_cast<int32_t>(H[q]);
        d.rounds = static_cast<int32_t>(R[q]);
        d.lo_iters = o.lo_iters;
        d.final_iters = o.final_iters;
        d.polish = o.p3p_fp64_polish;
        d.enumerate_all = o.enumerate_all;
        d.lo_fp64 = o.lo_fp64_accumulate;
        d.lo_solve64 = o.lo_fp64_solve;
        d.p_miss = o.p_miss;
        d.seed = o.seed;
        d.query_id = o.query_id;
        d.n_cap = static_cast<int32_t>(std::min<int64_t>(h.n_cap, INT32_MAX));
        d.inject = h.inject ? 1 : 0;
        const int64_t slots = std::max<int64_t>(1, max_wave_samples[q] * 4);
        d.subset = static_cast<ScorePair*>(ws_alloc(ctx, sizeof(ScorePair) * ((std::max(1, o.max_score_corr) + 1) / 2)));
        d.tc_mode = kTcVariants[tc_variant(ctx)].mode;
        if (bf16_on) {
            d.score_bf16 = 1;
            d.subset_b = static_cast<ScorePairB*>(
                ws_alloc(ctx, sizeof(ScorePairB) * (1 + (std::max(1, o.max_score_corr) + 1) / 2)));
            if (!d.subset_b) return IMLOC_ERR_OOM;
        }
        if (tc_on) {
            const int64_t mp = (std::max(1, o.max_score_corr) + kTcBlock - 1) / kTcBlock * kTcBlock;
            d.tc_rec = static_cast<float4*>(ws_alloc(ctx, 128 * mp));
            d.tc_e = d.tc_rec ? static_cast<float4*>(ws_alloc(ctx, 16 * mp)) : nullptr;
            if (!d.tc_e) {
                d.tc_rec = nullptr;
                tc_on = false;  // no room: every query of the call takes the FP32 scoring kernel
            }
        }
        if (h.slots_out) d.slots = h.slots_out;
        else d.slots = static_cast<PoseF*>(ws_alloc(ctx, sizeof(PoseF) * slots));
        d.compact = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * slots));
        if (h.round_best_out) d.round_best = h.round_best_out;
        else d.round_best = static_cast<uint64_t*>(ws_alloc(ctx, sizeof(uint64_t) * std::max<int64_t>(1, R[q])));
        d.round_hyps = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(1, R[q])));
        d.score_by_id = h.score_by_id;
        d.count_by_id = h.count_by_id;
        d.triples = h.triples;
        if (!d.subset || !d.slots || !d.compact || !d.round_best || !d.round_hyps) return IMLOC_ERR_OOM;
        est_hyp += h.inject ? H[q] : (H[q] * 3) / 2;
    }
    // fixed-set indices: share one buffer per concatenated correspondence set
    for (int q = 0; q < nq; ++q) {
        if (hq[q].fixidx_base) { qd[q].fixidx = hq[q].fixidx_base; continue; }
        bool shared = false;
        for (int p = 0; p < q; ++p)
            if (hq[p].X == hq[q].X && hq[p].d_off && hq[p].d_off == hq[q].d_off) { qd[q].fixidx = qd[p].fixidx; shared = true; break; }
        if (!shared) {
            qd[q].fixidx = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * std::max<int64_t>(1, hq[q].n_cap)));
            if (!qd[q].fixidx) return IMLOC_ERR_OOM;
        }
    }
    const size_t qd_bytes = sizeof(QueryDesc) * nq, wq_bytes = sizeof(WaveQ) * wq.size(),
                 wp_bytes = sizeof(int64_t) * wprefix.size();
    char* h_blk = static_cast<char*>(staging_alloc(ctx, qd_bytes + wq_bytes + wp_bytes + 512));
    char* d_blk = static_cast<char*>(ws_alloc(ctx, qd_bytes + wq_bytes + wp_bytes + 512));
    QueryState* d_qs = static_cast<QueryState*>(ws_alloc(ctx, sizeof(QueryState) * nq));
    int32_t* d_nhyp = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * W * nq));
    int32_t* d_tiles = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * (3 * nq + 1)));
    uint32_t* d_counter = static_cast<uint32_t*>(ws_alloc(ctx, sizeof(uint32_t)));
    if (!h_blk || !d_blk || !d_qs || !d_nhyp || !d_tiles || !d_counter) return IMLOC_ERR_OOM;
    const size_t o_wq = align_up(qd_bytes, 256), o_wp = align_up(o_wq + wq_bytes, 256);
    memcpy(h_blk, qd.data(), qd_bytes);
    memcpy(h_blk + o_wq, wq.data(), wq_bytes);
    memcpy(h_blk + o_wp, wprefix.data(), wp_bytes);
    int rc = upload(ctx, d_blk, h_blk, o_wp + wp_bytes, stream);
    if (rc != IMLOC_OK) return rc;
    const QueryDesc* d_qd = reinterpret_cast<const QueryDesc*>(d_blk);
    const WaveQ* d_wq = reinterpret_cast<const WaveQ*>(d_blk + o_wq);
    const int64_t* d_wp = reinterpret_cast<const int64_t*>(d_blk + o_wp);

    // injected poses go straight into the slots (one pose per sample)
    for (int q = 0; q < nq; ++q)
        if (hq[q].inject) {
            // slot of pose id 4 s is 4 s (single wave)
            IMLOC_CUDA_TRY(cudaMemcpy2DAsync(qd[q].slots, 4 * sizeof(PoseF), hq[q].inject, sizeof(PoseF), sizeof(PoseF),
                                             hq[q].n_inject, cudaMemcpyDeviceToDevice, stream));
        }

    // ---- launches: replayed from a CUDA graph per size bucket when possible ----
    // The workspace is carved in the same order for the same sizes, so equal
    // (query count, samples per wave, variant, buffers) give equal launches.
    const bool debug = hq[0].score_by_id || hq[0].count_by_id || hq[0].triples || hq[0].slots_out || hq[0].inject;
    // capture needs a real stream that nobody is capturing already (not the legacy default stream)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool real_stream = stream != nullptr && stream != cudaStreamLegacy && stream != cudaStreamPerThread &&
                             cudaStreamIsCapturing(stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    cudaGetLastError();
    // (the FP32 kernel's autotuner times launches: no capture before it has run)
    const bool use_graph = real_stream && !ctx->prof_on && (ctx->score_variant >= 0 || tc_on) && !debug &&
                           !getenv("IMLOC_NO_GRAPHS");
    std::string key;
    bool any_fp64 = false;  // FP64-accumulation queries add a replay launch: part of the bucket key
    for (int q = 0; q < nq; ++q) any_fp64 |= hq[q].o.lo_fp64_accumulate != 0;
    if (use_graph) {
        char buf[160];
        snprintf(buf, sizeof(buf), "%d|%d|%d|%d|%d|%d|%d|%p|%p|%p|%p|%p", nq, W, int(want_counts), int(any_fp64),
                 ctx->score_variant,
                 int(getenv("IMLOC_NO_FUSE") != nullptr) + 2 * int(getenv("IMLOC_FUSE") != nullptr),
                 bf16_on ? -1 : (tc_on ? 1 + tc_variant(ctx) : 0),
                 (const void*)d_qd, (void*)d_qs, (void*)d_nhyp, (void*)d_tiles, (const void*)d_wq);
        key = buf;
        for (int w = 0; w < W; ++w) key += "|" + std::to_string(wtotal[w]);
        auto it = ctx->graphs.find(key);
        if (it != ctx->graphs.end()) {
            IMLOC_CUDA_TRY(cudaGraphLaunch(it->second, stream));
            return IMLOC_OK;
        }
        if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            key.clear();
        }
    }
    const bool capturing = !key.empty();
    for (int w = 0; w < W; ++w) {
        StepBuffers sb;
        sb.d_qd = const_cast<QueryDesc*>(d_qd);
        sb.d_qs = d_qs;
        sb.d_wq = d_wq + static_cast<size_t>(w) * nq;
        sb.d_prefix = d_wp + static_cast<size_t>(w) * (nq + 1);
        sb.d_nhyp = d_nhyp + static_cast<size_t>(w) * nq;
        sb.d_tiles = d_tiles;
        sb.d_counter = d_counter;
        sb.d_nhyp_all = d_nhyp;
        sb.nhyp_all_len = W * nq;
        sb.d_init = nullptr;
        sb.any_fp64 = any_fp64;
        sb.fuse = dflt_fuse;
        sb.tc = tc_on;
        sb.bf16 = bf16_on;
        sb.d_rescored = reinterpret_cast<unsigned long long*>(hq[0].rescored_out);
        rc = run_step(ctx, sb, nq, w == 0 ? nq : 0, wtotal[w], want_counts, stream);
        if (rc != IMLOC_OK) {
            if (capturing) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(stream, &g);
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
            }
            return rc;
        }
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        IMLOC_CUDA_TRY(cudaStreamEndCapture(stream, &g));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        IMLOC_CUDA_TRY(e);
        if (ctx->graphs.size() >= 64) {
            for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
            ctx->graphs.clear();
        }
        ctx->graphs[key] = ge;
        IMLOC_CUDA_TRY(cudaGraphLaunch(ge, stream));
    }
    return IMLOC_OK;
}

}  // namespace imloc

// ============================================================================
// C ABI
// ============================================================================
using imloc::HostQuery;

static void fill_hostquery_from_corr(HostQuery& h, const imloc_corr* corr) {
    memset(&h, 0, sizeof(h));
    h.x = corr->x; h.y = corr->y; h.X = corr->X; h.Y = corr->Y; h.Z = corr->Z; h.w = corr->w;
    h.d_count = corr->count;
    h.n_host = corr->capacity;
    h.n_cap = corr->capacity;
}

extern "C" {

int imloc_ransac_pnp(imloc_ctx* ctx, const imloc_corr* corr, const imloc_camera* qcam, const imloc_ransac_opts* opts,
                     imloc_result* out, uint8_t* d_inlier_mask, void* stream) {
    if (!ctx || !corr || !qcam || !opts || !out) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = imloc::begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    imloc_result* d_res = static_cast<imloc_result*>(imloc::ws_alloc(ctx, sizeof(imloc_result)));
    if (!d_res) return IMLOC_ERR_OOM;
    HostQuery h;
    fill_hostquery_from_corr(h, corr);
    h.mask = d_inlier_mask;
    h.d_result = d_res;
    h.cam = *qcam;
    h.o = *opts;
    rc = imloc::ransac_impl(ctx, 1, &h, st, false);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaMemcpyAsync(out, d_res, sizeof(imloc_result), cudaMemcpyDeviceToHost, st));
    rc = imloc::end_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaStreamSynchronize(st));
    return out->status == IMLOC_OK ? IMLOC_OK : out->status;
}

int imloc_ransac_pnp_batch_async(imloc_ctx* ctx, int32_t n_queries, const imloc_corr* corr, const int64_t* d_offsets,
                                 const imloc_camera* qcams, const imloc_ransac_opts* opts, imloc_result* d_results,
                                 uint8_t* d_masks, void* stream) {
    if (!ctx || !corr || !d_offsets || !qcams || !opts || !d_results || n_queries <= 0) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = imloc::begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    std::vector<HostQuery> hq(n_queries);
    for (int q = 0; q < n_queries; ++q) {
        fill_hostquery_from_corr(hq[q], corr);
        hq[q].d_count = nullptr;
        hq[q].d_off = d_offsets;
        hq[q].q_off = q;
        hq[q].mask = d_masks;
        hq[q].d_result = d_results + q;
        hq[q].cam = qcams[q];
        hq[q].o = opts[q];
    }
    rc = imloc::ransac_impl(ctx, n_queries, hq.data(), st, false);
    int rc2 = imloc::end_call(ctx, st);
    return rc != IMLOC_OK ? rc : rc2;
}

int imloc_set_scoring(imloc_ctx* ctx, int32_t kernel, int32_t tc_variant) {
    if (!ctx || kernel < -1 || kernel > 1 || tc_variant < -1 || tc_variant >= imloc::kNumTcVariants)
        return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->scoring_kernel = kernel;
    ctx->scoring_tc_variant = tc_variant;
    return IMLOC_OK;
}

int imloc_score_config(const imloc_ctx* ctx, int32_t* threads, int32_t* poses_per_thread, int32_t* tile_poses) {
    if (!ctx) return IMLOC_ERR_INVALID_ARG;
    const int v = ctx->score_variant;
    if (v < 0 || v >= imloc::kNumScoreVariants) return IMLOC_ERR_NOT_FOUND;
    const imloc::ScoreVariant& V = imloc::kScoreVariants[v];
    if (threads) *threads = V.threads;
    if (poses_per_thread) *poses_per_thread = V.ht;
    if (tile_poses) *tile_poses = V.threads * V.ht;
    return IMLOC_OK;
}

int imloc_testing_ransac(imloc_ctx* ctx, const imloc_corr* corr, const imloc_camera* qcam,
                         const imloc_ransac_opts* opts, const imloc_debug* dbg, imloc_result* out,
                         uint8_t* d_inlier_mask, void* stream) {
    if (!ctx || !corr || !qcam || !opts || !out || !dbg) return IMLOC_ERR_INVALID_ARG;
    if (opts->p_miss > 0.0) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = imloc::begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    imloc_result* d_res = static_cast<imloc_result*>(imloc::ws_alloc(ctx, sizeof(imloc_result)));
    if (!d_res) return IMLOC_ERR_OOM;
    HostQuery h;
    fill_hostquery_from_corr(h, corr);
    h.d_count = nullptr;
    h.mask = d_inlier_mask;
    h.d_result = d_res;
    h.cam = *qcam;
    h.o = *opts;
    h.inject = reinterpret_cast<const imloc::PoseF*>(dbg->inject_poses);
    h.n_inject = dbg->inject_poses ? dbg->n_inject : 0;
    if (dbg->inject_poses && dbg->n_inject <= 0) return IMLOC_ERR_INVALID_ARG;
    h.score_by_id = dbg->scores;
    h.count_by_id = dbg->counts;
    h.triples = dbg->triples;
    h.slots_out = reinterpret_cast<imloc::PoseF*>(dbg->poses);
    h.round_best_out = dbg->round_best;
    h.rescored_out = dbg->rescored_pairs;
    rc = imloc::ransac_impl(ctx, 1, &h, st, dbg->counts != nullptr);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaMemcpyAsync(out, d_res, sizeof(imloc_result), cudaMemcpyDeviceToHost, st));
    rc = imloc::end_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaStreamSynchronize(st));
    return IMLOC_OK;
}

}  // extern "C"
