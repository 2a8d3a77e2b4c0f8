// rig.cu -- LO-RANSAC of the generalized absolute pose of a multi-camera rig
// (ImLoc supplementary "LaMAR HoloLens Results": queries taken by a camera
// rig, a GPU generalized absolute pose estimator).  The loop is that of
// Sec. 3.3 "Pose Estimation" with a generalized minimal solver and every
// residual taken in the camera that observed the point:
//   rig pose (rig_from_world) X_r = R X_w + t; camera k: X_c = R_k X_r + t_k.
//
// Kernels (per wave of rounds, all queries of the batch in each launch):
//   k_rig_setup   per query: N, the subset (uniform stride) regrouped by
//                 camera with a stable counting sort, round words
//   k_rig_sample  one minimal sample per thread: Philox triple, the three
//                 rays in the rig frame, the GP3P octic (gp3p.cuh, FP64) and
//                 its root brackets, appended to a list
//   k_rig_solve   one root bracket per thread: the root, back-substitution,
//                 Newton polish, the pose into slot 8 s + k (k = the root's
//                 rank in its sample), a compact list of the valid slots
//   k_rig_score   (query, tile of 128 poses, chunk of 1,024 subset records)
//                 per CTA, one pose per thread: the chunk staged in shared
//                 memory, per camera run the poses composed with that camera
//                 (K_k [R_k R | R_k t + t_k], FP32); partial truncated cost
//                 and inlier count per (pose, chunk)
//   k_rig_reduce  per pose: the partials in chunk order, one 64-bit atomic
//                 min into its round word
//   k_rig_replay  one cluster of CTAs per query: the rounds of the wave in order (new best
//                 -> LO on the subset), the adaptive stop, and once a query is
//                 done the final Cauchy refinement over all its
//                 correspondences; Gauss-Newton passes reduce FP32 per-thread
//                 sums in FP64 across warps, the 6x6 step is solved in FP64
// The host runs waves of 1, 1, 2, 4, 8, 8, ... rounds until every query is
// done (one 4-byte read-back per wave).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/imloc_testing.h"
#include "common.cuh"
#include "ctx.h"
#include "gp3p.cuh"

namespace imloc {

namespace {

constexpr int kRigMaxCams = IMLOC_RIG_MAX_CAMERAS;
constexpr int kRigSlots = 8;           // GP3P solutions per minimal sample
constexpr int kRigSampleThreads = 128;
constexpr int kRigScoreThreads = 128;
constexpr int kRigHT = 1;              // poses per scoring thread
constexpr int kRigTile = kRigScoreThreads * kRigHT;
constexpr int kRigChunk = 1024;        // subset records per scoring CTA (staged in shared memory)
constexpr int kRigReplayThreads = 512;
constexpr int kRigMaxWaveRounds = 8;

struct RigCam {
    float fx, fy, cx, cy;
    float R[9], t[3];      // cam_from_rig
    double Rd[9], td[3];
    double o[3];           // camera centre in the rig frame, -R^T t
};

struct RigBracket {
    double l, u, pl;     // root bracket of the sample's octic
    int32_t sl, k;       // sample within the wave, rank of the root
};

struct RigQuery {
    const float *x, *y, *X, *Y, *Z, *w;
    const int32_t* cam;
    const int64_t* d_off;
    int32_t q, n_cams;
    RigCam cams[kRigMaxCams];
    float tau2, cauchy2;
    int32_t m_cap, batch, rounds, lo_iters, final_iters, n_cap;
    int64_t max_iters;
    double p_miss;
    uint64_t seed;
    uint32_t query_id;
    int32_t pad0;
    imloc_result* result;
    uint8_t* mask;
    // workspace
    float4* rec;         // m_cap: X, Y, Z, w of the subset, grouped by camera
    float2* recxy;       // m_cap: observed pixel
    int32_t* seg;        // n_cams + 1 segment starts
    PoseF* slots;        // wave samples * 8
    int32_t* compact;    // wave samples * 8: valid slots of the wave
    int32_t* n_compact;
    RigBracket* brk;     // wave samples * 8 root brackets
    int32_t* n_brk;
    float2* part;        // wave samples * 8 * chunks: partial (cost, count bits) per pose and chunk
    uint64_t* round_best;
    int32_t* round_hyps;
    uint8_t* fix;        // fixed set of the final refinement, at the correspondences' offsets
    // test mode
    const PoseF* inject; // one pose per sample instead of GP3P (slot 8 s)
    int64_t n_inject;
    float* score_by_id;
    int32_t* count_by_id;
    int32_t* triples;
};

struct RigState {
    int64_t off, n;
    int32_t m, done, finished, status;
    double R[9], t[3];
    double best_score;
    int32_t have_best, subset_inliers, lo_count, rounds_done, passes, pad;
    int64_t best_hyp, iters, hypotheses;
};

struct RigWave {
    const RigQuery* qd;
    RigState* qs;
    int32_t* active;     // queries not finished
    int32_t r0, r1;      // rounds [r0, r1): samples [r0 batch, r1 batch) of each query
    int32_t final_wave;  // no rounds remain after this wave
    int32_t pad;
};

// ============================================================================
// setup
// ============================================================================
__global__ void __launch_bounds__(1024) k_rig_setup(const RigQuery* __restrict__ qd, RigState* qs) {
    const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const RigQuery& d = qd[q];
    __shared__ int64_t s_off, s_n;
    __shared__ int32_t s_m, s_bad;
    __shared__ int32_t s_cnt[kRigMaxCams], s_base[kRigMaxCams], s_seg[kRigMaxCams + 1];
    __shared__ int32_t s_wcnt[kRigMaxCams][32];
    if (tid == 0) {
        const int64_t off = d.d_off[d.q];
        int64_t n = d.d_off[d.q + 1] - off;
        RigState st;
        memset(&st, 0, sizeof(st));
        st.status = IMLOC_OK;
        if (n < 0 || off < 0 || off + n > d.n_cap) {
            n = 0;
            st.status = IMLOC_ERR_CAPACITY;
        }
        st.off = n > 0 ? off : 0;
        st.n = n;
        st.m = static_cast<int32_t>(n < d.m_cap ? n : d.m_cap);
        st.best_score = INFINITY;
        st.best_hyp = -1;
        qs[q] = st;
        s_off = st.off;
        s_n = n;
        s_m = st.m;
        s_bad = 0;
    }
    if (tid < kRigMaxCams) s_cnt[tid] = 0;
    for (int r = tid; r < d.rounds; r += blockDim.x) {
        d.round_best[r] = ~0ull;
        d.round_hyps[r] = 0;
    }
    __syncthreads();
    const int64_t off = s_off, n = s_n;
    const int m = s_m;
    // every camera index in range (the refinement reads all of them)
    for (int64_t i = off + tid; i < off + n; i += blockDim.x) {
        const int c = __ldg(d.cam + i);
        if (c < 0 || c >= d.n_cams) s_bad = 1;
    }
    // counting sort of the subset by camera (stable: subset order within a camera)
    for (int k = tid; k < m; k += blockDim.x) {
        const int c = __ldg(d.cam + off + (static_cast<int64_t>(k) * n) / m);
        if (c >= 0 && c < d.n_cams) atomicAdd(&s_cnt[c], 1);
    }
    __syncthreads();
    if (tid == 0) {
        s_seg[0] = 0;
        for (int c = 0; c < d.n_cams; ++c) {
            s_seg[c + 1] = s_seg[c] + s_cnt[c];
            s_base[c] = 0;
        }
        for (int c = 0; c <= d.n_cams; ++c) d.seg[c] = s_seg[c];
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            qs[q].status = IMLOC_ERR_INVALID_ARG;
            qs[q].done = 1;
        }
        return;
    }
    for (int k0 = 0; k0 < m; k0 += blockDim.x) {
        const int k = k0 + tid;
        int c = -1;
        int64_t i = 0;
        if (k < m) {
            i = off + (static_cast<int64_t>(k) * n) / m;
            c = __ldg(d.cam + i);
        }
        int my_rank = 0;
        for (int cc = 0; cc < d.n_cams; ++cc) {
            const uint32_t bal = __ballot_sync(0xffffffffu, c == cc);
            if (c == cc) my_rank = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) s_wcnt[cc][warp] = __popc(bal);
        }
        __syncthreads();
        if (c >= 0) {
            int before = 0;
            for (int w = 0; w < warp; ++w) before += s_wcnt[c][w];
            const int pos = s_seg[c] + s_base[c] + before + my_rank;
            d.rec[pos] = make_float4(__ldg(d.X + i), __ldg(d.Y + i), __ldg(d.Z + i), __ldg(d.w + i));
            d.recxy[pos] = make_float2(__ldg(d.x + i), __ldg(d.y + i));
        }
        __syncthreads();
        if (tid < d.n_cams) {
            int tot = 0;
            for (int w = 0; w < (blockDim.x >> 5); ++w) tot += s_wcnt[tid][w];
            s_base[tid] += tot;
        }
        __syncthreads();
    }
    if (tid == 0 && (n < 3 || d.rounds <= 0)) {
        qs[q].done = 1;
        if (qs[q].status == IMLOC_OK) qs[q].status = IMLOC_ERR_DEGENERATE;
    }
}

// ============================================================================
// minimal samples + GP3P
// ============================================================================
__device__ __forceinline__ void rig_ray(const RigQuery& d, int64_t i, double o[3], double dir[3], double X[3]) {
    const int k = __ldg(d.cam + i);
    const RigCam& c = d.cams[k];
    const double bx = (static_cast<double>(__ldg(d.x + i)) - c.cx) / c.fx;
    const double by = (static_cast<double>(__ldg(d.y + i)) - c.cy) / c.fy;
    const double inv = 1.0 / sqrt(bx * bx + by * by + 1.0);
    const double b[3] = {bx * inv, by * inv, inv};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dir[a] = c.Rd[a] * b[0] + c.Rd[3 + a] * b[1] + c.Rd[6 + a] * b[2];
        o[a] = c.o[a];
    }
    X[0] = __ldg(d.X + i);
    X[1] = __ldg(d.Y + i);
    X[2] = __ldg(d.Z + i);
}

// Phase 1, one thread per minimal sample: the triple, the rays, the GP3P
// coefficients and the root brackets over the whole grid, appended to the
// query's bracket list with their rank k (ascending lambda_1).
__global__ void __launch_bounds__(kRigSampleThreads) k_rig_sample(const __grid_constant__ RigWave w) {
    const int q = blockIdx.y;
    const RigQuery& d = w.qd[q];
    const RigState& st = w.qs[q];
    const int sl = blockIdx.x * kRigSampleThreads + threadIdx.x;
    if (sl >= (w.r1 - w.r0) * d.batch || st.done) return;
    const int64_t s = static_cast<int64_t>(w.r0) * d.batch + sl;
    if (s >= d.max_iters) return;
    if (d.inject) {  // test mode: the given pose, id 8 s
        if (s >= d.n_inject) return;
        d.slots[static_cast<int64_t>(sl) * kRigSlots] = d.inject[s];
        const int at = atomicAdd(d.n_compact, 1);
        d.compact[at] = sl * kRigSlots;
        atomicAdd(d.round_hyps + static_cast<int>(s / d.batch), 1);
        return;
    }
    int tri[3];
    const bool ok = draw_triple(d.seed, d.query_id, static_cast<uint32_t>(s), static_cast<uint32_t>(st.m), tri);
    if (d.triples) {
#pragma unroll
        for (int k = 0; k < 3; ++k) d.triples[3 * s + k] = ok ? tri[k] : -1;
    }
    if (!ok) return;
    double o[3][3], dir[3][3], X[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) rig_ray(d, st.off + (static_cast<int64_t>(tri[k]) * st.n) / st.m, o[k], dir[k], X[k]);
    Gp3pSys S;
    if (!gp3p_setup(o, dir, X, S)) return;
    Gp3pBracket br[kRigSlots];
    const int nb = gp3p_brackets(S, br, kRigSlots);
    if (nb == 0) return;
    const int at = atomicAdd(d.n_brk, nb);
    for (int k = 0; k < nb; ++k) d.brk[at + k] = RigBracket{br[k].l, br[k].u, br[k].pl, sl, k};
}

// Phase 2, one thread per root bracket: the sample's system again, the root,
// back-substitution and Newton polish, the pose into slot 8 s + k.
__global__ void __launch_bounds__(kRigSampleThreads) k_rig_solve(const __grid_constant__ RigWave w) {
    const int q = blockIdx.y;
    const RigQuery& d = w.qd[q];
    const RigState& st = w.qs[q];
    const int i = blockIdx.x * kRigSampleThreads + threadIdx.x;
    if (st.done || i >= *d.n_brk) return;
    const RigBracket b = d.brk[i];
    const int64_t s = static_cast<int64_t>(w.r0) * d.batch + b.sl;
    int tri[3];
    draw_triple(d.seed, d.query_id, static_cast<uint32_t>(s), static_cast<uint32_t>(st.m), tri);
    double o[3][3], dir[3][3], X[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) rig_ray(d, st.off + (static_cast<int64_t>(tri[k]) * st.n) / st.m, o[k], dir[k], X[k]);
    Gp3pSys S;
    gp3p_setup(o, dir, X, S);
    double L[3];
    if (!gp3p_finish(S, o, dir, Gp3pBracket{b.l, b.u, b.pl}, L)) return;
    double P[3][3], R[9], t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) P[k][a] = o[k][a] + L[k] * dir[k][a];
    if (!gp_pose(X, P, R, t)) return;
    PoseF pf;
#pragma unroll
    for (int a = 0; a < 9; ++a) pf.R[a] = static_cast<float>(R[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a) pf.t[a] = static_cast<float>(t[a]);
    const int slot = b.sl * kRigSlots + b.k;
    d.slots[slot] = pf;
    const int at = atomicAdd(d.n_compact, 1);
    d.compact[at] = slot;
    atomicAdd(d.round_hyps + static_cast<int>(s / d.batch), 1);
}

// ============================================================================
// scoring
// ============================================================================
// One CTA per (query, tile of kRigTile poses, chunk of kRigChunk subset
// records): the chunk is staged in shared memory once; for each camera run in
// it the poses are composed with that camera and evaluated on its records.
// Partial sums go to part[pose][chunk] (added in chunk order by k_rig_reduce:
// deterministic).
__global__ void __launch_bounds__(kRigScoreThreads) k_rig_score(const __grid_constant__ RigWave w) {
    const int q = blockIdx.z, tid = threadIdx.x;
    const RigQuery& d = w.qd[q];
    const int n_valid = *d.n_compact;
    const int base = blockIdx.x * kRigTile;
    const int m = w.qs[q].m;
    const int c0 = blockIdx.y * kRigChunk;
    if (base >= n_valid || c0 >= m || w.qs[q].done) return;
    const int c1 = min(m, c0 + kRigChunk);
    const int n_chunks = (m + kRigChunk - 1) / kRigChunk;
    __shared__ float4 s_rec[kRigChunk];
    __shared__ float2 s_xy[kRigChunk];
    __shared__ int32_t s_seg[kRigMaxCams + 1];
    if (tid <= d.n_cams) s_seg[tid] = d.seg[tid];
    for (int i = tid; i < c1 - c0; i += kRigScoreThreads) {
        s_rec[i] = d.rec[c0 + i];
        s_xy[i] = d.recxy[c0 + i];
    }
    int idx[kRigHT];
    float R[kRigHT][9], t[kRigHT][3];
#pragma unroll
    for (int j = 0; j < kRigHT; ++j) {
        idx[j] = base + j * kRigScoreThreads + tid;
        const int slot = idx[j] < n_valid ? d.compact[idx[j]] : d.compact[0];
        const PoseF p = d.slots[slot];
#pragma unroll
        for (int a = 0; a < 9; ++a) R[j][a] = p.R[a];
#pragma unroll
        for (int a = 0; a < 3; ++a) t[j][a] = p.t[a];
    }
    float cost[kRigHT];
    int cnt[kRigHT];
#pragma unroll
    for (int j = 0; j < kRigHT; ++j) {
        cost[j] = 0.f;
        cnt[j] = 0;
    }
    const float tau2 = d.tau2;
    __syncthreads();
    for (int k = 0; k < d.n_cams; ++k) {
        const int b0 = max(s_seg[k], c0), b1 = min(s_seg[k + 1], c1);
        if (b1 <= b0) continue;
        const RigCam& c = d.cams[k];
        // P_j = K_k [R_k R_j | R_k t_j + t_k]
        float P[kRigHT][12];
#pragma unroll
        for (int j = 0; j < kRigHT; ++j) {
            float M[3][4];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
                for (int bb = 0; bb < 3; ++bb)
                    M[a][bb] = fmaf(c.R[3 * a], R[j][bb], fmaf(c.R[3 * a + 1], R[j][3 + bb], c.R[3 * a + 2] * R[j][6 + bb]));
                M[a][3] = fmaf(c.R[3 * a], t[j][0], fmaf(c.R[3 * a + 1], t[j][1], fmaf(c.R[3 * a + 2], t[j][2], c.t[a])));
            }
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                P[j][bb] = fmaf(c.fx, M[0][bb], c.cx * M[2][bb]);
                P[j][4 + bb] = fmaf(c.fy, M[1][bb], c.cy * M[2][bb]);
                P[j][8 + bb] = M[2][bb];
            }
        }
        // two records of the run per step, their projections and residuals as
        // packed f32x2 operations (the pose coefficients duplicated in both
        // halves), branch-free: z <= 0 (or NaN) gives 1/0 = inf, an inf or
        // NaN residual, min(., tau^2) = tau^2 and no inlier; the even and the
        // odd records are summed separately, then even + odd
        uint64_t P2[kRigHT][12];
#pragma unroll
        for (int j = 0; j < kRigHT; ++j)
#pragma unroll
            for (int a = 0; a < 12; ++a) P2[j][a] = f2_pack(P[j][a], P[j][a]);
        float pe[kRigHT], po[kRigHT];
#pragma unroll
        for (int j = 0; j < kRigHT; ++j) { pe[j] = 0.f; po[j] = 0.f; }
        const int i0 = b0 - c0, i1 = b1 - c0;
        int i = i0;
#pragma unroll 2
        for (; i + 2 <= i1; i += 2) {
            const float4 A = s_rec[i], B = s_rec[i + 1];
            const float2 xa = s_xy[i], xb = s_xy[i + 1];
            const uint64_t X2 = f2_pack(A.x, B.x), Y2 = f2_pack(A.y, B.y), Z2 = f2_pack(A.z, B.z);
            const uint64_t NX = f2_pack(-xa.x, -xb.x), NY = f2_pack(-xa.y, -xb.y);
#pragma unroll
            for (int j = 0; j < kRigHT; ++j) {
                const uint64_t zu = f2_fma(P2[j][0], X2, f2_fma(P2[j][1], Y2, f2_fma(P2[j][2], Z2, P2[j][3])));
                const uint64_t zv = f2_fma(P2[j][4], X2, f2_fma(P2[j][5], Y2, f2_fma(P2[j][6], Z2, P2[j][7])));
                const uint64_t zz = f2_fma(P2[j][8], X2, f2_fma(P2[j][9], Y2, f2_fma(P2[j][10], Z2, P2[j][11])));
                float z0, z1;
                f2_unpack(zz, z0, z1);
                const uint64_t iz = f2_pack(rcp_approx(fmaxf(z0, 0.0f)), rcp_approx(fmaxf(z1, 0.0f)));
                const uint64_t du = f2_fma(zu, iz, NX), dv = f2_fma(zv, iz, NY);
                float r0, r1;
                f2_unpack(f2_fma(du, du, f2_mul(dv, dv)), r0, r1);
                cnt[j] += ((r0 < tau2) ? 1 : 0) + ((r1 < tau2) ? 1 : 0);
                pe[j] = fmaf(A.w, fminf(r0, tau2), pe[j]);
                po[j] = fmaf(B.w, fminf(r1, tau2), po[j]);
            }
        }
        if (i < i1) {  // odd run length: the last record alone
            const float4 X = s_rec[i];
            const float2 xy = s_xy[i];
#pragma unroll
            for (int j = 0; j < kRigHT; ++j) {
                const float u = fmaf(P[j][0], X.x, fmaf(P[j][1], X.y, fmaf(P[j][2], X.z, P[j][3])));
                const float v = fmaf(P[j][4], X.x, fmaf(P[j][5], X.y, fmaf(P[j][6], X.z, P[j][7])));
                const float z = fmaf(P[j][8], X.x, fmaf(P[j][9], X.y, fmaf(P[j][10], X.z, P[j][11])));
                const float iz = rcp_approx(fmaxf(z, 0.0f));
                const float du = fmaf(u, iz, -xy.x), dv = fmaf(v, iz, -xy.y);
                const float rr = fmaf(du, du, dv * dv);
                cnt[j] += (rr < tau2) ? 1 : 0;
                pe[j] = fmaf(X.w, fminf(rr, tau2), pe[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kRigHT; ++j) cost[j] += pe[j] + po[j];
    }
#pragma unroll
    for (int j = 0; j < kRigHT; ++j)
        if (idx[j] < n_valid)
            d.part[static_cast<int64_t>(idx[j]) * n_chunks + blockIdx.y] = make_float2(cost[j], __int_as_float(cnt[j]));
}

// Per valid pose: the chunk partial sums in chunk order, its score and count,
// and the 64-bit atomic min (score bits << 32 | pose id) into its round word.
__global__ void __launch_bounds__(256) k_rig_reduce(const __grid_constant__ RigWave w) {
    const int q = blockIdx.y;
    const RigQuery& d = w.qd[q];
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= *d.n_compact || w.qs[q].done) return;
    const int m = w.qs[q].m;
    const int n_chunks = (m + kRigChunk - 1) / kRigChunk;
    float cost = 0.f;
    int cnt = 0;
    for (int c = 0; c < n_chunks; ++c) {
        const float2 pc = d.part[static_cast<int64_t>(i) * n_chunks + c];
        cost += pc.x;
        cnt += __float_as_int(pc.y);
    }
    const int64_t gid = static_cast<int64_t>(w.r0) * d.batch * kRigSlots + d.compact[i];  // 8 * sample + solution
    if (d.score_by_id) d.score_by_id[gid] = cost;
    if (d.count_by_id) d.count_by_id[gid] = cnt;
    const int r = static_cast<int>((gid / kRigSlots) / d.batch);
    const uint64_t key = (static_cast<uint64_t>(__float_as_uint(cost)) << 32) | static_cast<uint32_t>(gid);
    atomicMin(reinterpret_cast<unsigned long long*>(d.round_best + r), static_cast<unsigned long long>(key));
}

// ============================================================================
// replay: rounds in order, LO, adaptive stop, final refinement
// ============================================================================
struct RigReplaySmem {
    double R[9], t[3];        // pose of the pass
    double Rc[9], tc[3];      // candidate pose
    double H[21], g[6], cost;
    double Hs[21], gs[6];     // normal equations of the current pose (damping retries)
    int32_t count, used;
    double wsum[kRigReplayThreads / 32][30];
    double part[2][32];          // this CTA's sums of a pass (read by the whole cluster), double-buffered
    int32_t pbuf;                // buffer of the next pass
    float Pc[kRigMaxCams][12];   // K_k [R_k R | R_k t + t_k] of the pass pose, FP32
    float Rk[kRigMaxCams][9];    // R_k
    float Rf[9], tf[3];          // pass pose, FP32
    int32_t seg[kRigMaxCams + 1];
    int32_t ok, stop;
    double step2;
};

enum { kLossTrunc = 0, kLossCauchy = 1 };
enum { kSrcSubset = 0, kSrcAll = 1, kSrcFixed = 2 };

// pixel Jacobian of the left perturbation of the rig pose, X_r' = Exp(w) X_r + v:
// dX_c/d(w, v) = R_k [-[X_r]_x | I]; J rows in a0 (u) and a1 (v)
__device__ __forceinline__ void rig_point_terms(const float Rk[9], float fx, float fy, const float Xr[3],
                                                const float Xc[3], float J0[6], float J1[6]) {
    const float iz = 1.0f / Xc[2];
    const float du0 = fx * iz, du2 = -fx * Xc[0] * iz * iz;
    const float dv1 = fy * iz, dv2 = -fy * Xc[1] * iz * iz;
    // a = dpi/dXc R_k (row vectors)
    float a0[3], a1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        a0[b] = fmaf(du0, Rk[b], du2 * Rk[6 + b]);
        a1[b] = fmaf(dv1, Rk[3 + b], dv2 * Rk[6 + b]);
    }
    // a (-[X_r]_x): columns (0, Z, -Y), (-Z, 0, X), (Y, -X, 0) of the skew form
    J0[0] = fmaf(-a0[1], Xr[2], a0[2] * Xr[1]);
    J0[1] = fmaf(a0[0], Xr[2], -a0[2] * Xr[0]);
    J0[2] = fmaf(-a0[0], Xr[1], a0[1] * Xr[0]);
    J1[0] = fmaf(-a1[1], Xr[2], a1[2] * Xr[1]);
    J1[1] = fmaf(a1[0], Xr[2], -a1[2] * Xr[0]);
    J1[2] = fmaf(-a1[0], Xr[1], a1[1] * Xr[0]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        J0[3 + b] = a0[b];
        J1[3 + b] = a1[b];
    }
}

// the FP32 per-camera matrices of the pose in S.R, S.t
__device__ void rig_set_pose(RigReplaySmem& S, const RigQuery& d) {
    const int tid = threadIdx.x;
    if (tid < d.n_cams) {
        const RigCam& c = d.cams[tid];
        double M[3][4];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b)
                M[a][b] = c.Rd[3 * a] * S.R[b] + c.Rd[3 * a + 1] * S.R[3 + b] + c.Rd[3 * a + 2] * S.R[6 + b];
            M[a][3] = c.Rd[3 * a] * S.t[0] + c.Rd[3 * a + 1] * S.t[1] + c.Rd[3 * a + 2] * S.t[2] + c.td[a];
        }
        for (int b = 0; b < 4; ++b) {
            S.Pc[tid][b] = static_cast<float>(c.fx * M[0][b] + c.cx * M[2][b]);
            S.Pc[tid][4 + b] = static_cast<float>(c.fy * M[1][b] + c.cy * M[2][b]);
            S.Pc[tid][8 + b] = static_cast<float>(M[2][b]);
        }
        for (int a = 0; a < 9; ++a) S.Rk[tid][a] = c.R[a];
    }
    if (tid < 9) S.Rf[tid] = static_cast<float>(S.R[tid]);
    if (tid < 3) S.tf[tid] = static_cast<float>(S.t[tid]);
    __syncthreads();
}

// One pass over the subset (grouped by camera), all correspondences, or the
// fixed set: cost (truncated or Cauchy), inliers, and with NORMAL the normal
// equations (points used: truncated -> inliers; Cauchy -> all in front).
// Sums: FP32 per thread and per warp, FP64 across warps.  Result in S.
template <int SRC, int LOSS, bool NORMAL>
__device__ void rig_pass(RigReplaySmem& S, const RigQuery& d, const RigState& st) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float acc[30];
#pragma unroll
    for (int k = 0; k < 30; ++k) acc[k] = 0.f;  // H[21], g[6], cost, count, used
    const float tau2 = d.tau2, c2 = d.cauchy2;
    auto point = [&](int k, float X, float Y, float Z, float wt, float x, float y) {
        const float* P = S.Pc[k];
        const float u = fmaf(P[0], X, fmaf(P[1], Y, fmaf(P[2], Z, P[3])));
        const float v = fmaf(P[4], X, fmaf(P[5], Y, fmaf(P[6], Z, P[7])));
        const float z = fmaf(P[8], X, fmaf(P[9], Y, fmaf(P[10], Z, P[11])));
        float rr = tau2;
        bool front = z > 0.f, in = false;
        float r0 = 0.f, r1 = 0.f;
        if (front) {
            const float iz = __frcp_rn(z);
            r0 = fmaf(u, iz, -x);
            r1 = fmaf(v, iz, -y);
            rr = fmaf(r0, r0, r1 * r1);
            in = rr < tau2;
        }
        if (LOSS == kLossTrunc) {
            acc[27] = fmaf(wt, in ? rr : tau2, acc[27]);
        } else {
            acc[27] = fmaf(wt * c2, log1pf((front ? rr : tau2) / c2), acc[27]);
        }
        acc[28] += in ? 1.f : 0.f;
        if (NORMAL) {
            const bool use = LOSS == kLossTrunc ? in : front;
            if (use) {
                const float ww = LOSS == kLossTrunc ? wt : wt / (1.f + rr / c2);
                const float Xr[3] = {fmaf(S.Rf[0], X, fmaf(S.Rf[1], Y, fmaf(S.Rf[2], Z, S.tf[0]))),
                                     fmaf(S.Rf[3], X, fmaf(S.Rf[4], Y, fmaf(S.Rf[5], Z, S.tf[1]))),
                                     fmaf(S.Rf[6], X, fmaf(S.Rf[7], Y, fmaf(S.Rf[8], Z, S.tf[2])))};
                const RigCam& c = d.cams[k];
                const float Xc[3] = {fmaf(S.Rk[k][0], Xr[0], fmaf(S.Rk[k][1], Xr[1], fmaf(S.Rk[k][2], Xr[2], c.t[0]))),
                                     fmaf(S.Rk[k][3], Xr[0], fmaf(S.Rk[k][4], Xr[1], fmaf(S.Rk[k][5], Xr[2], c.t[1]))),
                                     fmaf(S.Rk[k][6], Xr[0], fmaf(S.Rk[k][7], Xr[1], fmaf(S.Rk[k][8], Xr[2], c.t[2])))};
                float J0[6], J1[6];
                rig_point_terms(S.Rk[k], c.fx, c.fy, Xr, Xc, J0, J1);
                int h = 0;
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const float wa0 = ww * J0[a], wa1 = ww * J1[a];
#pragma unroll
                    for (int b = a; b < 6; ++b) acc[h++] += fmaf(wa0, J0[b], wa1 * J1[b]);
                    acc[21 + a] += fmaf(wa0, r0, wa1 * r1);
                }
                acc[29] += 1.f;
            }
        }
    };
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = static_cast<int>(cluster.block_rank()), ncl = static_cast<int>(cluster.num_blocks());
    const int stride = ncl * kRigReplayThreads, first = rank * kRigReplayThreads + tid;
    if (SRC == kSrcSubset) {
        for (int k = 0; k < d.n_cams; ++k)
            for (int i = S.seg[k] + first; i < S.seg[k + 1]; i += stride) {
                const float4 X = d.rec[i];
                const float2 xy = d.recxy[i];
                point(k, X.x, X.y, X.z, X.w, xy.x, xy.y);
            }
    } else {
        for (int64_t i = st.off + first; i < st.off + st.n; i += stride) {
            if (SRC == kSrcFixed && !d.fix[i]) continue;
            point(__ldg(d.cam + i), __ldg(d.X + i), __ldg(d.Y + i), __ldg(d.Z + i), __ldg(d.w + i), __ldg(d.x + i),
                  __ldg(d.y + i));
        }
    }
    if (NORMAL) {
        // butterfly reduce-scatter across the warp: after the 5 steps lane l holds
        // the warp's total of value l (31 shuffles for 32 values instead of 5 each)
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = k < 30 ? acc[k] : 0.f;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const float send = upper ? v[i] : v[i + o];
                const float keep = upper ? v[i + o] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        if (lane < 30) S.wsum[warp][lane] = v[0];
    } else {
#pragma unroll
        for (int k = 27; k < 30; ++k) {
            float v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) S.wsum[warp][k] = v;
        }
    }
    // cluster sums through a double-buffered array: a CTA writes buffer pb of
    // this pass while a slower CTA may still read the other one from the last
    const int pb = S.pbuf;
    __syncthreads();
    if (tid < 30 && (NORMAL || tid >= 27)) {
        double s = 0.0;
        for (int w = 0; w < kRigReplayThreads / 32; ++w) s += S.wsum[w][tid];
        S.part[pb][tid] = s;
    }
    cluster.sync();
    // every CTA of the cluster adds the CTAs' sums in rank order: identical totals
    if (tid < 30 && (NORMAL || tid >= 27)) {
        double s = 0.0;
        for (int r = 0; r < ncl; ++r) s += cluster.map_shared_rank(&S.part[pb][0], r)[tid];
        if (tid < 21) S.H[tid] = s;
        else if (tid < 27) S.g[tid - 21] = s;
        else if (tid == 27) S.cost = s;
        else if (tid == 28) S.count = static_cast<int32_t>(s + 0.5);
        else S.used = static_cast<int32_t>(s + 0.5);
    }
    __syncthreads();
    if (tid == 0) S.pbuf = pb ^ 1;
    __syncthreads();
}

__device__ bool rig_solve6(const double Hu[21], const double g[6], double mu, double x[6]) {
    double A[6][6];
    int h = 0;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) {
            A[a][b] = A[b][a] = Hu[h++];
        }
    for (int a = 0; a < 6; ++a) A[a][a] += mu * A[a][a];
    double L[6][6] = {{0}};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    double z[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
        z[i] = s / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return true;
}

// candidate = Exp(w) [R | t] + v (Rodrigues, FP64)
__device__ void rig_apply(const double dl[6], const double R[9], const double t[3], double Rn[9], double tn[3]) {
    const double th2 = dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2];
    const double th = sqrt(th2);
    double A, B;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0, -dl[2], dl[1], dl[2], 0, -dl[0], -dl[1], dl[0], 0};
    double E[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double K2 = 0.0;
            for (int k = 0; k < 3; ++k) K2 += K[3 * i + k] * K[3 * k + j];
            E[3 * i + j] = (i == j ? 1.0 : 0.0) + A * K[3 * i + j] + B * K2;
        }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Rn[3 * i + j] = E[3 * i] * R[j] + E[3 * i + 1] * R[3 + j] + E[3 * i + 2] * R[6 + j];
        tn[i] = E[3 * i] * t[0] + E[3 * i + 1] * t[1] + E[3 * i + 2] * t[2] + dl[3 + i];
    }
}

// Gauss-Newton with the schedule of the single-camera loop: steps kept only if
// the cost drops (Marquardt damping 0, 1e-3, 1e-2, 1e-1 of diag H), stop on a
// step below 1e-10 or a decrease below 1e-6 of the cost.  Pose in S.R/S.t.
// Each pass at a candidate also forms its normal equations, so an accepted
// step costs one pass (the equations of the next step are already there).
template <int SRC, int LOSS>
__device__ double rig_gauss_newton(RigReplaySmem& S, const RigQuery& d, RigState& st, int iters) {
    const int tid = threadIdx.x;
    rig_set_pose(S, d);
    rig_pass<SRC, LOSS, true>(S, d, st);
    double cost = S.cost;
    if (tid == 0) st.passes += 1;
    for (int it = 0; it < iters; ++it) {
        if (S.used < 3) break;
        __syncthreads();
        if (tid < 21) S.Hs[tid] = S.H[tid];
        if (tid < 6) S.gs[tid] = S.g[tid];
        const double R0[9] = {S.R[0], S.R[1], S.R[2], S.R[3], S.R[4], S.R[5], S.R[6], S.R[7], S.R[8]};
        const double t0[3] = {S.t[0], S.t[1], S.t[2]};
        bool ok = false;
        double mu = 0.0, cn = cost, step2 = 0.0;
        for (int attempt = 0; attempt < 4; ++attempt) {
            __syncthreads();
            if (tid == 0) {
                double dl[6];
                S.ok = rig_solve6(S.Hs, S.gs, mu, dl);
                if (S.ok) {
                    rig_apply(dl, R0, t0, S.R, S.t);
                    double n2 = 0.0;
                    for (int k = 0; k < 6; ++k) n2 += dl[k] * dl[k];
                    S.step2 = n2;
                }
            }
            __syncthreads();
            if (S.ok) {
                rig_set_pose(S, d);
                rig_pass<SRC, LOSS, true>(S, d, st);
                if (tid == 0) st.passes += 1;
                cn = S.cost;
                step2 = S.step2;
                if (cn < cost) {
                    ok = true;
                    break;
                }
            }
            mu = (mu == 0.0) ? 1e-3 : mu * 10.0;
        }
        __syncthreads();
        if (!ok) {
            // keep the pose before the rejected attempts
            if (tid < 9) S.R[tid] = R0[tid];
            if (tid < 3) S.t[tid] = t0[tid];
            __syncthreads();
            break;
        }
        const double decrease = cost - cn;
        const bool converged = sqrt(step2) < 1e-10 || decrease < 1e-6 * cost;
        cost = cn;
        if (converged) break;
    }
    return cost;
}

// nearest rotation of a nearly orthonormal R (from float32): Newton-Schulz
// steps R <- R (3 I - R^T R) / 2, quadratic convergence
__device__ void rig_orthonormalize(double R[9]) {
    for (int it = 0; it < 4; ++it) {
        double A[9], N[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                A[3 * i + j] = R[i] * R[j] + R[3 + i] * R[3 + j] + R[6 + i] * R[6 + j];  // R^T R
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                N[3 * i + j] = 0.5 * (3.0 * R[3 * i + j] -
                                      (R[3 * i] * A[j] + R[3 * i + 1] * A[3 + j] + R[3 * i + 2] * A[6 + j]));
        for (int k = 0; k < 9; ++k) R[k] = N[k];
    }
}

__device__ double rig_needed_iters(double eps, double p_miss) {
    const double e3 = eps * eps * eps;
    if (e3 >= 1.0) return 0.0;
    if (e3 <= 0.0) return INFINITY;
    return log(p_miss) / log(1.0 - e3);
}

// One cluster of CTAs per query: every CTA runs the same decisions on the
// same cluster-reduced sums; the points of each pass are split across the
// CTAs; rank 0 writes the state and the result.
__global__ void __launch_bounds__(kRigReplayThreads) k_rig_replay(const __grid_constant__ RigWave w) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = static_cast<int>(cluster.block_rank()), ncl = static_cast<int>(cluster.num_blocks());
    const int q = blockIdx.x / ncl, tid = threadIdx.x;
    const bool lead = rank == 0 && tid == 0;
    const int first = rank * kRigReplayThreads + tid, stride = ncl * kRigReplayThreads;
    const RigQuery& d = w.qd[q];
    __shared__ RigReplaySmem S;
    __shared__ RigState st;
    if (tid == 0) {
        st = w.qs[q];
        S.pbuf = 0;
    }
    if (tid <= kRigMaxCams) S.seg[tid] = tid <= d.n_cams ? d.seg[tid] : 0;
    cluster.sync();  // every CTA has read the state before rank 0 may write it
    if (st.finished) return;
    const int64_t rounds_total = (d.max_iters + d.batch - 1) / d.batch;
    if (!st.done) {
        const int r_end = min(w.r1, d.rounds);  // queries may have fewer rounds than the longest
        for (int r = w.r0; r < r_end; ++r) {
            const uint64_t key = d.round_best[r];
            const float sc = __uint_as_float(static_cast<uint32_t>(key >> 32));
            __syncthreads();
            if (key != ~0ull && static_cast<double>(sc) < st.best_score) {
                const int64_t gid = static_cast<int64_t>(key & 0xffffffffu);
                const PoseF p = d.slots[gid - static_cast<int64_t>(w.r0) * d.batch * kRigSlots];
                if (tid == 0) {
                    for (int a = 0; a < 9; ++a) S.R[a] = p.R[a];
                    for (int a = 0; a < 3; ++a) S.t[a] = p.t[a];
                    rig_orthonormalize(S.R);
                }
                __syncthreads();
                double best = sc;
                if (tid == 0) {
                    st.best_score = sc;
                    st.best_hyp = gid;
                    st.have_best = 1;
                }
                if (d.lo_iters > 0) {
                    const double R0[9] = {S.R[0], S.R[1], S.R[2], S.R[3], S.R[4], S.R[5], S.R[6], S.R[7], S.R[8]};
                    const double t0[3] = {S.t[0], S.t[1], S.t[2]};
                    const double lc = rig_gauss_newton<kSrcSubset, kLossTrunc>(S, d, st, d.lo_iters);
                    __syncthreads();
                    if (tid == 0) st.lo_count += 1;
                    if (lc < best) {
                        best = lc;
                    } else {
                        if (tid < 9) S.R[tid] = R0[tid];
                        if (tid < 3) S.t[tid] = t0[tid];
                    }
                    __syncthreads();
                }
                if (tid == 0) {
                    st.best_score = best;
                    for (int a = 0; a < 9; ++a) st.R[a] = S.R[a];
                    for (int a = 0; a < 3; ++a) st.t[a] = S.t[a];
                }
                rig_set_pose(S, d);
                rig_pass<kSrcSubset, kLossTrunc, false>(S, d, st);
                if (tid == 0) st.subset_inliers = S.count;
            }
            __syncthreads();
            if (tid == 0) {
                st.iters = min(static_cast<int64_t>(r + 1) * d.batch, d.max_iters);
                st.rounds_done = r + 1;
                st.hypotheses += d.round_hyps[r];
                if (st.iters >= d.max_iters) st.done = 1;
                else if (d.p_miss > 0.0 && st.have_best &&
                         static_cast<double>(st.iters) >=
                             rig_needed_iters(static_cast<double>(st.subset_inliers) / st.m, d.p_miss))
                    st.done = 1;
            }
            __syncthreads();
            if (st.done) break;
        }
        if (tid == 0 && !st.done && (st.rounds_done >= rounds_total || w.final_wave)) st.done = 1;
        __syncthreads();
    }
    if (!st.done) {
        if (lead) w.qs[q] = st;
        return;
    }
    // final refinement over all correspondences: fixed set = inliers of the best model
    imloc_result* res = d.result;
    if (st.have_best) {
        if (tid < 9) S.R[tid] = st.R[tid];
        if (tid < 3) S.t[tid] = st.t[tid];
        __syncthreads();
        rig_set_pose(S, d);
        const float tau2 = d.tau2;
        for (int64_t i = st.off + first; i < st.off + st.n; i += stride) {
            const int k = __ldg(d.cam + i);
            const float* P = S.Pc[k];
            const float X = __ldg(d.X + i), Y = __ldg(d.Y + i), Z = __ldg(d.Z + i);
            const float u = fmaf(P[0], X, fmaf(P[1], Y, fmaf(P[2], Z, P[3])));
            const float v = fmaf(P[4], X, fmaf(P[5], Y, fmaf(P[6], Z, P[7])));
            const float z = fmaf(P[8], X, fmaf(P[9], Y, fmaf(P[10], Z, P[11])));
            bool in = false;
            if (z > 0.f) {
                const float iz = __frcp_rn(z);
                const float r0 = fmaf(u, iz, -__ldg(d.x + i)), r1 = fmaf(v, iz, -__ldg(d.y + i));
                in = fmaf(r0, r0, r1 * r1) < tau2;
            }
            d.fix[i] = in ? 1 : 0;  // read back by this CTA only (same partition)
        }
        __syncthreads();
        if (d.final_iters > 0) rig_gauss_newton<kSrcFixed, kLossCauchy>(S, d, st, d.final_iters);
        __syncthreads();
        rig_set_pose(S, d);
        // inliers of the final pose over all correspondences (and the mask)
        int cnt = 0;
        for (int64_t i = st.off + first; i < st.off + st.n; i += stride) {
            const int k = __ldg(d.cam + i);
            const float* P = S.Pc[k];
            const float X = __ldg(d.X + i), Y = __ldg(d.Y + i), Z = __ldg(d.Z + i);
            const float u = fmaf(P[0], X, fmaf(P[1], Y, fmaf(P[2], Z, P[3])));
            const float v = fmaf(P[4], X, fmaf(P[5], Y, fmaf(P[6], Z, P[7])));
            const float z = fmaf(P[8], X, fmaf(P[9], Y, fmaf(P[10], Z, P[11])));
            bool in = false;
            if (z > 0.f) {
                const float iz = __frcp_rn(z);
                const float r0 = fmaf(u, iz, -__ldg(d.x + i)), r1 = fmaf(v, iz, -__ldg(d.y + i));
                in = fmaf(r0, r0, r1 * r1) < tau2;
            }
            if (d.mask) d.mask[i] = in ? 1 : 0;
            cnt += in;
        }
        cnt = warp_sum_i(cnt);
        if ((tid & 31) == 0) S.wsum[tid >> 5][0] = cnt;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w2 = 0; w2 < kRigReplayThreads / 32; ++w2) tot += S.wsum[w2][0];
            S.part[S.pbuf][0] = tot;
        }
        cluster.sync();
        if (lead) {
            double tot = 0.0;
            for (int r2 = 0; r2 < ncl; ++r2) tot += cluster.map_shared_rank(&S.part[S.pbuf][0], r2)[0];
            imloc_result r;
            memset(&r, 0, sizeof(r));
            for (int a = 0; a < 9; ++a) {
                r.R[a] = S.R[a];
                r.R_best[a] = st.R[a];
            }
            for (int a = 0; a < 3; ++a) {
                r.t[a] = S.t[a];
                r.t_best[a] = st.t[a];
            }
            r.score = st.best_score;
            r.num_inliers = static_cast<int64_t>(tot + 0.5);
            r.subset_inliers = st.subset_inliers;
            r.iterations = st.iters;
            r.rounds = st.rounds_done;
            r.lo_count = st.lo_count;
            r.hypotheses = st.hypotheses;
            r.best_hyp = st.best_hyp;
            r.status = st.status;
            r.passes = st.passes;
            *res = r;
        }
    } else {
        if (d.mask)
            for (int64_t i = st.off + first; i < st.off + st.n; i += stride) d.mask[i] = 0;
        if (lead) {
            imloc_result r;
            memset(&r, 0, sizeof(r));
            r.iterations = st.iters;
            r.rounds = st.rounds_done;
            r.hypotheses = st.hypotheses;
            r.best_hyp = -1;
            r.status = st.status != IMLOC_OK ? st.status : IMLOC_ERR_DEGENERATE;
            *res = r;
        }
    }
    if (lead) {
        st.finished = 1;
        w.qs[q] = st;
        atomicSub(w.active, 1);
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// ============================================================================
// host
// ============================================================================
struct RigHostQuery {
    const imloc_rig* rig;
    imloc_ransac_opts o;
    imloc_result* d_result;
    uint8_t* mask;
    const PoseF* inject;
    int64_t n_inject;
    float* score_by_id;
    int32_t* count_by_id;
    int32_t* triples;
    PoseF* slots_out;
    uint64_t* round_best_out;
};

template <typename K, typename P>
int rig_launch_cluster(K kernel, const P& params, int grid, int block, int cluster, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
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

bool rig_ok(const imloc_rig& r) {
    if (r.n_cams < 1 || r.n_cams > kRigMaxCams) return false;
    for (int k = 0; k < r.n_cams; ++k) {
        const imloc_camera& c = r.cams[k];
        if (!(c.fx != 0.f) || !(c.fy != 0.f) || !isfinite(c.fx) || !isfinite(c.fy) || !isfinite(c.cx) ||
            !isfinite(c.cy))
            return false;
        for (int a = 0; a < 9; ++a)
            if (!isfinite(r.cam_from_rig[k].R[a])) return false;
        for (int a = 0; a < 3; ++a)
            if (!isfinite(r.cam_from_rig[k].t[a])) return false;
    }
    return true;
}

int rig_impl(imloc_ctx* ctx, int nq, const imloc_corr* corr, const int32_t* d_cam, const int64_t* d_offsets,
             const RigHostQuery* hq, cudaStream_t st, bool single_wave) {
    if (!corr->x || !corr->y || !corr->X || !corr->Y || !corr->Z || !corr->w || !d_cam || !d_offsets)
        return IMLOC_ERR_INVALID_ARG;
    int max_rounds = 0;
    for (int q = 0; q < nq; ++q) {
        const imloc_ransac_opts& o = hq[q].o;
        if (!hq[q].rig || !rig_ok(*hq[q].rig)) return IMLOC_ERR_INVALID_ARG;
        if (!(o.tau_px > 0.0) || o.max_score_corr < 3 || o.batch <= 0 || o.max_iters <= 0 ||
            o.max_iters > (1 << 28) || o.lo_iters < 0 || o.final_iters < 0 || o.enumerate_all != 0)
            return IMLOC_ERR_INVALID_ARG;
        max_rounds = std::max(max_rounds, (o.max_iters + o.batch - 1) / o.batch);
    }
    // waves: 1, 1, 2, 4, 8, 8, ... rounds (all rounds at once in single-wave mode)
    std::vector<std::pair<int, int>> waves;
    {
        int r = 0, len = 1, k = 0;
        while (r < max_rounds) {
            const int l = single_wave ? max_rounds : std::min(len, max_rounds - r);
            waves.push_back({r, r + l});
            r += l;
            if (k++ >= 1) len = std::min(len * 2, kRigMaxWaveRounds);
        }
    }
    int wave_rounds = 0;
    for (auto& wv : waves) wave_rounds = std::max(wave_rounds, wv.second - wv.first);
    // replay: a cluster of up to 8 CTAs per query while the batch leaves SMs free
    int replay_cl = 8;
    while (replay_cl > 1 && static_cast<int64_t>(nq) * replay_cl > ctx->sm_count) replay_cl >>= 1;
    int max_batch = 0, max_chunks = 1;
    for (int q = 0; q < nq; ++q) {
        max_batch = std::max(max_batch, hq[q].o.batch);
        max_chunks = std::max(max_chunks, (hq[q].o.max_score_corr + kRigChunk - 1) / kRigChunk);
    }
    const int64_t wave_samples = static_cast<int64_t>(wave_rounds) * max_batch;

    RigQuery* hd = static_cast<RigQuery*>(staging_alloc(ctx, sizeof(RigQuery) * nq));
    RigQuery* dd = static_cast<RigQuery*>(ws_alloc(ctx, sizeof(RigQuery) * nq));
    RigState* qs = static_cast<RigState*>(ws_alloc(ctx, sizeof(RigState) * nq));
    int32_t* active = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t)));
    int32_t* h_active = static_cast<int32_t*>(staging_alloc(ctx, sizeof(int32_t)));
    uint8_t* fix = static_cast<uint8_t*>(ws_alloc(ctx, static_cast<size_t>(std::max<int64_t>(corr->capacity, 1))));
    int32_t* n_compact = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * 2 * nq));  // poses, brackets
    if (!hd || !dd || !qs || !active || !h_active || !fix || !n_compact) return IMLOC_ERR_OOM;
    for (int q = 0; q < nq; ++q) {
        const imloc_ransac_opts& o = hq[q].o;
        const imloc_rig& rg = *hq[q].rig;
        RigQuery& d = hd[q];
        memset(&d, 0, sizeof(d));
        d.x = corr->x;
        d.y = corr->y;
        d.X = corr->X;
        d.Y = corr->Y;
        d.Z = corr->Z;
        d.w = corr->w;
        d.cam = d_cam;
        d.d_off = d_offsets;
        d.q = q;
        d.n_cams = rg.n_cams;
        for (int k = 0; k < rg.n_cams; ++k) {
            RigCam& c = d.cams[k];
            c.fx = rg.cams[k].fx;
            c.fy = rg.cams[k].fy;
            c.cx = rg.cams[k].cx;
            c.cy = rg.cams[k].cy;
            for (int a = 0; a < 9; ++a) {
                c.Rd[a] = rg.cam_from_rig[k].R[a];
                c.R[a] = static_cast<float>(c.Rd[a]);
            }
            for (int a = 0; a < 3; ++a) {
                c.td[a] = rg.cam_from_rig[k].t[a];
                c.t[a] = static_cast<float>(c.td[a]);
            }
            for (int a = 0; a < 3; ++a) c.o[a] = -(c.Rd[a] * c.td[0] + c.Rd[3 + a] * c.td[1] + c.Rd[6 + a] * c.td[2]);
        }
        d.tau2 = static_cast<float>(o.tau_px * o.tau_px);
        const double cs = o.cauchy_scale > 0.0 ? o.cauchy_scale : o.tau_px;
        d.cauchy2 = static_cast<float>(cs * cs);
        d.m_cap = o.max_score_corr;
        d.batch = o.batch;
        d.rounds = (o.max_iters + o.batch - 1) / o.batch;
        d.lo_iters = o.lo_iters;
        d.final_iters = o.final_iters;
        d.n_cap = static_cast<int32_t>(std::min<int64_t>(corr->capacity, 0x7fffffff));
        d.max_iters = o.max_iters;
        d.p_miss = o.p_miss;
        d.seed = o.seed;
        d.query_id = o.query_id;
        d.result = hq[q].d_result;
        d.mask = hq[q].mask;
        d.rec = static_cast<float4*>(ws_alloc(ctx, sizeof(float4) * o.max_score_corr));
        d.recxy = static_cast<float2*>(ws_alloc(ctx, sizeof(float2) * o.max_score_corr));
        d.seg = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * (kRigMaxCams + 1)));
        d.slots = hq[q].slots_out ? hq[q].slots_out
                                  : static_cast<PoseF*>(ws_alloc(ctx, sizeof(PoseF) * wave_samples * kRigSlots));
        d.compact = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * wave_samples * kRigSlots));
        d.n_compact = n_compact + q;
        d.n_brk = n_compact + nq + q;
        d.brk = static_cast<RigBracket*>(ws_alloc(ctx, sizeof(RigBracket) * wave_samples * kRigSlots));
        d.part = static_cast<float2*>(ws_alloc(ctx, sizeof(float2) * wave_samples * kRigSlots *
                                                         ((o.max_score_corr + kRigChunk - 1) / kRigChunk)));
        d.round_best = hq[q].round_best_out
                           ? hq[q].round_best_out
                           : static_cast<uint64_t*>(ws_alloc(ctx, sizeof(uint64_t) * std::max(1, d.rounds)));
        d.round_hyps = static_cast<int32_t*>(ws_alloc(ctx, sizeof(int32_t) * std::max(1, d.rounds)));
        d.fix = fix;
        d.inject = hq[q].inject;
        d.n_inject = hq[q].n_inject;
        d.score_by_id = hq[q].score_by_id;
        d.count_by_id = hq[q].count_by_id;
        d.triples = hq[q].triples;
        if (!d.rec || !d.recxy || !d.seg || !d.slots || !d.compact || !d.brk || !d.part || !d.round_best ||
            !d.round_hyps)
            return IMLOC_ERR_OOM;
    }
    *h_active = nq;
    int rc = upload(ctx, dd, hd, sizeof(RigQuery) * nq, st);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaMemcpyAsync(active, h_active, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    {
        ProfScope prof(ctx, st, "k_rig_setup");
        k_rig_setup<<<nq, 1024, 0, st>>>(dd, qs);
        IMLOC_CUDA_TRY(cudaGetLastError());
        prof.end();
    }
    for (size_t wi = 0; wi < waves.size(); ++wi) {
        RigWave w;
        w.qd = dd;
        w.qs = qs;
        w.active = active;
        w.r0 = waves[wi].first;
        w.r1 = waves[wi].second;
        w.final_wave = wi + 1 == waves.size();
        w.pad = 0;
        const int64_t ns = static_cast<int64_t>(w.r1 - w.r0) * max_batch;  // samples of the largest batch
        IMLOC_CUDA_TRY(cudaMemsetAsync(n_compact, 0, sizeof(int32_t) * 2 * nq, st));
        {
            ProfScope prof(ctx, st, "k_rig_sample");
            k_rig_sample<<<dim3(static_cast<unsigned>((ns + kRigSampleThreads - 1) / kRigSampleThreads), nq),
                           kRigSampleThreads, 0, st>>>(w);
            IMLOC_CUDA_TRY(cudaGetLastError());
            prof.end();
        }
        {
            ProfScope prof(ctx, st, "k_rig_solve");
            k_rig_solve<<<dim3(static_cast<unsigned>((ns * kRigSlots + kRigSampleThreads - 1) / kRigSampleThreads), nq),
                          kRigSampleThreads, 0, st>>>(w);
            IMLOC_CUDA_TRY(cudaGetLastError());
            prof.end();
        }
        {
            const int tiles = static_cast<int>((ns * kRigSlots + kRigTile - 1) / kRigTile);
            ProfScope prof(ctx, st, "k_rig_score");
            k_rig_score<<<dim3(tiles, max_chunks, nq), kRigScoreThreads, 0, st>>>(w);
            IMLOC_CUDA_TRY(cudaGetLastError());
            prof.end();
        }
        {
            ProfScope prof(ctx, st, "k_rig_reduce");
            k_rig_reduce<<<dim3(static_cast<unsigned>((ns * kRigSlots + 255) / 256), nq), 256, 0, st>>>(w);
            IMLOC_CUDA_TRY(cudaGetLastError());
            prof.end();
        }
        {
            ProfScope prof(ctx, st, "k_rig_replay");
            rc = rig_launch_cluster(k_rig_replay, w, nq * replay_cl, kRigReplayThreads, replay_cl, st);
            if (rc != IMLOC_OK) return rc;
            prof.end();
        }
        if (w.final_wave) break;
        IMLOC_CUDA_TRY(cudaMemcpyAsync(h_active, active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        IMLOC_CUDA_TRY(cudaStreamSynchronize(st));
        if (*h_active <= 0) break;
    }
    return IMLOC_OK;
}

}  // namespace

}  // namespace imloc

extern "C" {

int imloc_ransac_rig_batch(imloc_ctx* ctx, int32_t n_queries, const imloc_corr* corr, const int32_t* d_cam,
                           const int64_t* d_offsets, const imloc_rig* rigs, const imloc_ransac_opts* opts,
                           imloc_result* d_results, uint8_t* d_masks, void* stream) {
    using namespace imloc;
    if (!ctx || n_queries < 1 || !corr || !d_cam || !d_offsets || !rigs || !opts || !d_results)
        return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    std::vector<RigHostQuery> hq(n_queries);
    for (int q = 0; q < n_queries; ++q) {
        RigHostQuery& h = hq[q];
        memset(&h, 0, sizeof(h));
        h.rig = &rigs[q];
        h.o = opts[q];
        h.d_result = d_results + q;
        h.mask = d_masks;
    }
    rc = rig_impl(ctx, n_queries, corr, d_cam, d_offsets, hq.data(), st, false);
    const int rc2 = end_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    if (rc2 != IMLOC_OK) return rc2;
    IMLOC_CUDA_TRY(cudaStreamSynchronize(st));
    return IMLOC_OK;
}

int imloc_testing_rig(imloc_ctx* ctx, const imloc_corr* corr, const int32_t* d_cam, const imloc_rig* rig,
                      const imloc_ransac_opts* opts, const imloc_debug* dbg, imloc_result* out,
                      uint8_t* d_inlier_mask, void* stream) {
    using namespace imloc;
    if (!ctx || !corr || !d_cam || !rig || !opts || !dbg || !out) return IMLOC_ERR_INVALID_ARG;
    if (opts->p_miss > 0.0) return IMLOC_ERR_INVALID_ARG;
    if (dbg->inject_poses && dbg->n_inject <= 0) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    imloc_result* d_res = static_cast<imloc_result*>(ws_alloc(ctx, sizeof(imloc_result)));
    int64_t* d_off = static_cast<int64_t*>(ws_alloc(ctx, sizeof(int64_t) * 2));
    int64_t* h_off = static_cast<int64_t*>(staging_alloc(ctx, sizeof(int64_t) * 2));
    if (!d_res || !d_off || !h_off) return IMLOC_ERR_OOM;
    h_off[0] = 0;
    h_off[1] = corr->capacity;
    rc = upload(ctx, d_off, h_off, sizeof(int64_t) * 2, st);
    if (rc != IMLOC_OK) return rc;
    const int64_t H = opts->max_iters;
    if (dbg->scores) IMLOC_CUDA_TRY(cudaMemsetAsync(dbg->scores, 0xff, sizeof(float) * H * kRigSlots, st));
    if (dbg->counts) IMLOC_CUDA_TRY(cudaMemsetAsync(dbg->counts, 0xff, sizeof(int32_t) * H * kRigSlots, st));
    if (dbg->poses) IMLOC_CUDA_TRY(cudaMemsetAsync(dbg->poses, 0xff, sizeof(PoseF) * H * kRigSlots, st));
    RigHostQuery h;
    memset(&h, 0, sizeof(h));
    h.rig = rig;
    h.o = *opts;
    h.d_result = d_res;
    h.mask = d_inlier_mask;
    h.inject = reinterpret_cast<const PoseF*>(dbg->inject_poses);
    h.n_inject = dbg->inject_poses ? dbg->n_inject : 0;
    h.score_by_id = dbg->scores;
    h.count_by_id = dbg->counts;
    h.triples = dbg->triples;
    h.slots_out = reinterpret_cast<PoseF*>(dbg->poses);
    h.round_best_out = dbg->round_best;
    rc = rig_impl(ctx, 1, corr, d_cam, d_off, &h, st, true);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaMemcpyAsync(out, d_res, sizeof(imloc_result), cudaMemcpyDeviceToHost, st));
    rc = end_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    IMLOC_CUDA_TRY(cudaStreamSynchronize(st));
    return IMLOC_OK;
}

}  // extern "C"
