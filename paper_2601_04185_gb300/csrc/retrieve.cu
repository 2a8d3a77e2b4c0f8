// retrieve.cu -- nearest-neighbour search of global retrieval features (ImLoc
// Sec. 3.1: per database image a precomputed global descriptor; Sec. 4.4
// "Runtime": the nearest-neighbour search of the retrieval features on the GPU).
//
// scores = DB x Q^T as a bf16 GEMM on the 5th-generation tensor cores:
// k_retrieve_gemm is persistent (one CTA per SM), with warp roles
//   warp 4      TMA producer: 128 database rows x 64 dims and Nq query rows
//               x 64 dims per pipeline stage (128-byte swizzle), mbarriers
//   warp 5      TMEM allocator and MMA issuer: 4 tcgen05.mma (M=128, N=Nq,
//               K=16) per stage into an FP32 accumulator in tensor memory,
//               double buffered so that the epilogue of one tile overlaps the
//               MMAs of the next
//   warps 0-3   epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32w..32w+31 = database rows), query-major score stores
// The database is the M side, so one kernel serves a single query (HBM-bound:
// every descriptor byte is read once) and batches of up to 256 queries
// (tensor-bound).  The top-K per query then comes from k_topk_select over
// 64-bit keys (orderable score bits, inverted index: ties go to the lower
// database index): partitions of up to 4,096 scores held in registers, a
// threshold that at least K keys reach (from the threads' maxima), the keys
// above it ranked exactly, and the partitions' lists merged by the last block
// of each query to finish.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "ctx.h"
#include "tc.cuh"

namespace imloc {

namespace {

constexpr int kTileM = 128;        // database rows per tile (TMEM lanes)
constexpr int kTileK = 64;         // bf16 dims per stage (one 128-byte swizzle row)
constexpr int kUmmaK = 16;         // K of one tcgen05.mma for 16-bit inputs
constexpr int kMaxNq = 256;        // queries per launch (MMA N)
constexpr int kGemmThreads = 192;  // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr int kSelectChunk = 4096; // scores (or candidates) one selection CTA holds
constexpr int kMaxK = 128;

struct GemmParams {
    CUtensorMap map_db;  // bf16 [N][D], box {64, 128}
    CUtensorMap map_q;   // bf16 [Q][D], box {64, Nq}
    float* scores;       // [Q][ld]
    int64_t ld;
    int64_t N;
    int32_t Q, D, Nq, stages, tmem_cols;
    int32_t n_tiles;
    int* err;
};

__device__ __forceinline__ uint32_t stage_bytes_a() { return kTileM * kTileK * 2; }

__global__ void __launch_bounds__(kGemmThreads, 1) k_retrieve_gemm(const __grid_constant__ GemmParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the swizzled stage buffers
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = p.stages, Nq = p.Nq;
    const uint32_t a_bytes = stage_bytes_a(), b_bytes = static_cast<uint32_t>(Nq) * kTileK * 2;
    unsigned char* sa = smem;
    unsigned char* sb = smem + static_cast<size_t>(S) * a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sb + static_cast<size_t>(S) * b_bytes);
    uint64_t* full = bars;              // [S]
    uint64_t* empty = bars + S;         // [S]
    uint64_t* tfull = bars + 2 * S;     // [2]
    uint64_t* tempty = bars + 2 * S + 2;// [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 128);
        }
        mbar_fence_init();
    }
    if (warp == 5) {
        tmem_alloc(tmem_slot, static_cast<uint32_t>(p.tmem_cols));
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int KB = (p.D + kTileK - 1) / kTileK;

    if (warp == 4) {
        if (lane == 0) {
            tma_prefetch_map(&p.map_db);
            tma_prefetch_map(&p.map_q);
            uint32_t it = 0;
            for (int t = blockIdx.x; t < p.n_tiles; t += gridDim.x) {
                const int m0 = t * kTileM;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = static_cast<int>(it % S);
                    const uint32_t ph = (it / S) & 1u;
                    mbar_wait_bounded(&empty[s], ph ^ 1u, p.err);
                    mbar_arrive_expect_tx(&full[s], a_bytes + b_bytes);
                    tma_load_2d(sa + static_cast<size_t>(s) * a_bytes, &p.map_db, kb * kTileK, m0, &full[s]);
                    tma_load_2d(sb + static_cast<size_t>(s) * b_bytes, &p.map_q, kb * kTileK, 0, &full[s]);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(kTileM, static_cast<uint32_t>(Nq));
            uint32_t it = 0, lt = 0;
            for (int t = blockIdx.x; t < p.n_tiles; t += gridDim.x, ++lt) {
                const uint32_t buf = lt & 1u;
                mbar_wait_bounded(&tempty[buf], ((lt >> 1) & 1u) ^ 1u, p.err);
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + buf * static_cast<uint32_t>(Nq);
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = static_cast<int>(it % S);
                    const uint32_t ph = (it / S) & 1u;
                    mbar_wait_bounded(&full[s], ph, p.err);
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sa + static_cast<size_t>(s) * a_bytes);
                    const uint32_t b0 = smem_u32(sb + static_cast<size_t>(s) * b_bytes);
#pragma unroll
                    for (int kk = 0; kk < kTileK / kUmmaK; ++kk) {
                        // K step of 16 bf16 = 32 bytes inside the swizzled 128-byte rows
                        const uint64_t ad = umma_desc_k_sw128(a0 + kk * kUmmaK * 2);
                        const uint64_t bd = umma_desc_k_sw128(b0 + kk * kUmmaK * 2);
                        umma_bf16(d_tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);  // frees the stage when these MMAs have read it
                }
                umma_commit(&tfull[buf]);    // accumulator complete
            }
        }
    } else {
        // epilogue: warp w owns TMEM lanes 32w..32w+31, i.e. database rows m0 + 32w + lane
        uint32_t lt = 0;
        for (int t = blockIdx.x; t < p.n_tiles; t += gridDim.x, ++lt) {
            const uint32_t buf = lt & 1u;
            mbar_wait_bounded(&tfull[buf], (lt >> 1) & 1u, p.err);
            tc_fence_after();
            const int64_t row = static_cast<int64_t>(t) * kTileM + warp * 32 + lane;
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(warp * 32) << 16) + buf * static_cast<uint32_t>(Nq);
            for (int c = 0; c < Nq; c += 16) {
                float v[16];
                tmem_ld_32x32b_x16(taddr + static_cast<uint32_t>(c), v);
                if (row < p.N) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c + j < p.Q) p.scores[static_cast<int64_t>(c + j) * p.ld + row] = v[j];
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[buf]);
        }
    }
    // every warp is done: the last MMAs completed before the epilogue read them
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem_base, static_cast<uint32_t>(p.tmem_cols));
    }
}

// ---- one or two queries: the search is a matrix-vector product, bound by
// reading the database once.  Each warp streams whole rows (16-byte loads,
// 8 in flight per lane, consecutive lanes on consecutive 16 bytes) against
// the queries held as FP32 in shared memory (two planes, so that the 16-byte
// shared loads of a warp are contiguous); per-lane FP32 sums in a fixed
// order, then a fixed shuffle tree: identical rows give identical scores.
constexpr int kGemvThreads = 512;
constexpr int kGemvMaxQ = 2;
constexpr int kGemvUnroll = 8;

struct GemvParams {
    const uint4* db;  // [N][D / 8]: 8 bf16 per uint4
    const uint4* q;   // [Q][D / 8]
    float* scores;    // [Q][ld]
    int64_t ld, N;
    int32_t D8, pad;
};

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

template <int Q>
__global__ void __launch_bounds__(kGemvThreads) k_retrieve_gemv(const __grid_constant__ GemvParams p) {
    extern __shared__ float4 s_q[];  // [Q][2][D8]: values 0-3 and 4-7 of each group of 8
    const int D8 = p.D8;
    for (int i = threadIdx.x; i < Q * D8; i += kGemvThreads) {
        const int qq = i / D8, j = i - qq * D8;
        const uint4 v = p.q[static_cast<int64_t>(qq) * D8 + j];
        s_q[(2 * qq) * D8 + j] = make_float4(bf16_lo(v.x), bf16_hi(v.x), bf16_lo(v.y), bf16_hi(v.y));
        s_q[(2 * qq + 1) * D8 + j] = make_float4(bf16_lo(v.z), bf16_hi(v.z), bf16_lo(v.w), bf16_hi(v.w));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (kGemvThreads / 32);
    for (int64_t row = static_cast<int64_t>(blockIdx.x) * (kGemvThreads / 32) + (threadIdx.x >> 5); row < p.N;
         row += nw) {
        const uint4* r = p.db + row * D8;
        float acc[Q];
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) acc[qq] = 0.f;
        for (int j0 = lane; j0 < D8; j0 += 32 * kGemvUnroll) {
            uint4 v[kGemvUnroll];
#pragma unroll
            for (int u = 0; u < kGemvUnroll; ++u) {
                const int j = j0 + 32 * u;
                v[u] = j < D8 ? __ldcs(r + j) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < kGemvUnroll; ++u) {
                const int j = j0 + 32 * u;
                if (j < D8) {
#pragma unroll
                    for (int qq = 0; qq < Q; ++qq) {
                        const float4 a = s_q[(2 * qq) * D8 + j], b = s_q[(2 * qq + 1) * D8 + j];
                        float t = acc[qq];
                        t = fmaf(bf16_lo(v[u].x), a.x, t);
                        t = fmaf(bf16_hi(v[u].x), a.y, t);
                        t = fmaf(bf16_lo(v[u].y), a.z, t);
                        t = fmaf(bf16_hi(v[u].y), a.w, t);
                        t = fmaf(bf16_lo(v[u].z), b.x, t);
                        t = fmaf(bf16_hi(v[u].z), b.y, t);
                        t = fmaf(bf16_lo(v[u].w), b.z, t);
                        t = fmaf(bf16_hi(v[u].w), b.w, t);
                        acc[qq] = t;
                    }
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[qq] += __shfl_xor_sync(0xffffffffu, acc[qq], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int qq = 0; qq < Q; ++qq) p.scores[qq * p.ld + row] = acc[qq];
        }
    }
}

// ---- top-K selection ---------------------------------------------------------
// key: orderable score bits << 32 | (0xffffffff - index): larger key = higher
// score, then lower index; 0 = padding (below every real key)
__device__ __forceinline__ uint64_t score_key(float s, uint32_t idx) {
    const uint32_t u = __float_as_uint(s);
    const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return (static_cast<uint64_t>(o) << 32) | (0xffffffffu - idx);
}
__device__ __forceinline__ float key_score(uint64_t k) {
    const uint32_t o = static_cast<uint32_t>(k >> 32);
    const uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}
__device__ __forceinline__ uint32_t key_index(uint64_t k) { return 0xffffffffu - static_cast<uint32_t>(k); }

struct SelectParams {
    const float* scores;     // level 0: [Q][ld] scores, N valid
    const uint64_t* keys_in; // later levels: [Q][L] keys
    int64_t ld;
    int64_t L;               // elements per query at this level (scores: N)
    uint64_t* keys_out;      // [Q][chunks * K] sorted keys per chunk (padding 0)
    int32_t K;
    int32_t chunks;          // per query
    int32_t chunk;           // elements per chunk (<= kSelectChunk)
    // final level (chunks * K <= kSelectChunk): the last block of a query to finish
    // merges the query's chunk lists and writes the result; null: another level follows
    uint32_t* tickets;       // [Q], zero at launch
    float* out_score;        // [Q][K], -inf past the N-th
    int32_t* out_index;      // [Q][K], -1 past the N-th
};

constexpr int kSelThreads = 256;
constexpr int kSelCand = 1024;  // candidates sorted exactly (the keys at or above the threshold)

constexpr int kSelWarps = kSelThreads / 32;
static_assert(kMaxK <= 32 * kSelWarps, "each warp's threshold rank must fit in a warp");

// Bitonic sort of one value a lane, descending from lane 0 (shuffles only).
__device__ __forceinline__ uint32_t warp_sort_desc(uint32_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool keep_max = ((lane & k) == 0) == ((lane & j) == 0);
            v = keep_max ? max(v, o) : min(v, o);
        }
    return v;
}

// Where a block's selected keys go: the next level's key list, or the result.
struct SelectOut {
    uint64_t* keys;   // K keys, 0 past the n-th; null: result
    float* score;     // K scores, -inf past the n-th
    int32_t* index;   // K database rows, -1 past the n-th
};

// Writes the n unique keys in cand (shared memory) in descending order: rank r
// = the number of keys that exceed it, kept for r < K.  Ranks are counted
// directly (n <= kSelCand): no sorting network, no barriers.
__device__ __forceinline__ void emit_ranked(const uint64_t* cand, int n, int K, const SelectOut& o, int tid) {
    for (int i = tid; i < n; i += kSelThreads) {
        const uint64_t k = cand[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += cand[j] > k;
        if (r < K) {
            if (o.keys) {
                o.keys[r] = k;
            } else {
                o.score[r] = key_score(k);
                o.index[r] = static_cast<int32_t>(key_index(k));
            }
        }
    }
    for (int i = n + tid; i < K; i += kSelThreads) {
        if (o.keys) {
            o.keys[i] = 0ull;
        } else {
            o.score[i] = -INFINITY;
            o.index[i] = -1;
        }
    }
}

// Scanning the histogram from its top bin down: the bin that holds the K-th
// counted element and the count in the bins above it.  Thread t owns the BPT
// contiguous bins from t*BPT; one warp-level suffix scan, no serial walk.  With
// fewer than K counted elements: bin 0 and the count above it.
template <int BPT>
__device__ __forceinline__ void hist_crossing(const uint32_t* hist, int K, int tid, uint32_t* s_wsum, int* s_bin,
                                              int* s_above) {
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t c[BPT];
    uint32_t own = 0u;
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
        c[j] = hist[tid * BPT + j];
        own += c[j];
    }
    uint32_t inc = own;  // inclusive suffix sum within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_down_sync(0xffffffffu, inc, o);
        if (lane + o < 32) inc += v;
    }
    if (lane == 0) s_wsum[warp] = inc;
    __syncthreads();
    uint32_t above = 0u, total = 0u;
#pragma unroll
    for (int w = 0; w < kSelThreads / 32; ++w) {
        total += s_wsum[w];
        if (w > warp) above += s_wsum[w];
    }
    uint32_t cnt = inc - own + above;  // elements in bins above this thread's range
    const uint32_t k = static_cast<uint32_t>(K);
    if (total < k) {
        if (tid == 0) {
            *s_bin = 0;
            *s_above = static_cast<int>(total - hist[0]);
        }
    } else if (cnt < k && cnt + own >= k) {
#pragma unroll
        for (int j = BPT - 1; j >= 0; --j) {
            if (cnt + c[j] >= k) {
                *s_bin = tid * BPT + j;
                *s_above = static_cast<int>(cnt);
                break;
            }
            cnt += c[j];
        }
    }
    __syncthreads();
}

// Exact top-K keys of one chunk of <= kSelectChunk elements, sorted descending,
// with the chunk held in registers (kSelEPT elements a thread).  Usually: the
// keys whose score bits reach the K-th largest thread maximum, collected and
// sorted.  When more than kSelCand keys reach it (ties, or data laid out in
// order): radix selection over the 64-bit keys.
//   kScores: level 0, the thread's elements are kSelEPT/4 float4 groups of the
//   score row (ld a multiple of 4); else keys of the previous level, 0 = empty.
constexpr int kSelEPT = kSelectChunk / kSelThreads;

struct SelectSmem {
    uint64_t cand[kSelCand];
    uint64_t prefix, mask;
    uint32_t hist[256];
    uint32_t wtau[kSelWarps], wsum[kSelWarps];
    int n, bstar, above, rem, done, last;
};

// One block's selection: the top K of the m elements from `sc` (kScores: a score
// row starting at database row b) or `kr` (a key list), written to `o`.
template <bool kScores>
__device__ __forceinline__ void select_block(SelectSmem& sm, const float* sc, const uint64_t* kr, int64_t b, int m,
                                             int Kmax, const SelectOut& o) {
    uint64_t* const s_cand = sm.cand;
    uint32_t* const s_hist = sm.hist;
    uint32_t* const s_wtau = sm.wtau;
    uint32_t* const s_wsum = sm.wsum;
    int& s_n = sm.n;
    int& s_bstar = sm.bstar;
    int& s_above = sm.above;
    int& s_rem = sm.rem;
    int& s_done = sm.done;
    uint64_t& s_prefix = sm.prefix;
    uint64_t& s_mask = sm.mask;
    const int tid = threadIdx.x, lane = tid & 31;
    auto pos = [&](int i) -> int {  // offset of the thread's element i in the chunk
        return kScores ? 4 * (tid + kSelThreads * (i >> 2)) + (i & 3) : tid + kSelThreads * i;
    };
    uint32_t hw[kSelEPT];                  // orderable score bits
    uint32_t lw[kScores ? 1 : kSelEPT];    // low key words (level 0: from the position)
    uint32_t valid = 0u;
    if constexpr (kScores) {
        lw[0] = 0u;
        const float* row = sc;
        float4 f[kSelEPT / 4];
#pragma unroll
        for (int j = 0; j < kSelEPT / 4; ++j) {  // independent loads, all in flight together
            const int e = pos(4 * j);
            f[j] = e + 3 < m ? *reinterpret_cast<const float4*>(row + e) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int j = 0; j < kSelEPT / 4; ++j) {
            const int e = pos(4 * j);
            if (e + 3 < m) {
                valid |= 0xfu << (4 * j);
            } else if (e < m) {  // the group holding the end of a ragged chunk
                f[j].x = row[e];
                f[j].y = e + 1 < m ? row[e + 1] : 0.0f;
                f[j].z = e + 2 < m ? row[e + 2] : 0.0f;
                valid |= ((1u << (m - e)) - 1u) << (4 * j);
            }
            hw[4 * j + 0] = static_cast<uint32_t>(score_key(f[j].x, 0u) >> 32);
            hw[4 * j + 1] = static_cast<uint32_t>(score_key(f[j].y, 0u) >> 32);
            hw[4 * j + 2] = static_cast<uint32_t>(score_key(f[j].z, 0u) >> 32);
            hw[4 * j + 3] = static_cast<uint32_t>(score_key(f[j].w, 0u) >> 32);
        }
    } else {
        // L2 loads: the lists may come from other blocks of this launch
        uint64_t k[kSelEPT];
#pragma unroll
        for (int i = 0; i < kSelEPT; ++i) k[i] = pos(i) < m ? __ldcg(kr + pos(i)) : 0ull;
#pragma unroll
        for (int i = 0; i < kSelEPT; ++i) {
            hw[i] = static_cast<uint32_t>(k[i] >> 32);
            lw[i] = static_cast<uint32_t>(k[i]);
            if (k[i] != 0ull) valid |= 1u << i;
        }
    }
    auto key = [&](int i) -> uint64_t {
        const uint32_t l = kScores ? 0xffffffffu - (static_cast<uint32_t>(b) + static_cast<uint32_t>(pos(i))) : lw[kScores ? 0 : i];
        return (static_cast<uint64_t>(hw[i]) << 32) | l;
    };
    const int K = min(Kmax, m);
    // Threshold tau: each warp sorts its threads' maxima (shuffles) and takes the
    // ceil(K/8)-th largest; tau is the smallest of the eight.  Every warp then
    // holds ceil(K/8) keys with score bits >= tau, so at least K keys reach it,
    // and for unordered data not many more do.
    uint32_t tmax = 0u;
#pragma unroll
    for (int i = 0; i < kSelEPT; ++i)
        if (valid & (1u << i)) tmax = max(tmax, hw[i]);
    const int kw = (K + kSelWarps - 1) / kSelWarps;
    const uint32_t tw = __shfl_sync(0xffffffffu, warp_sort_desc(tmax, lane), kw > 0 ? kw - 1 : 0);
    if (lane == 0) s_wtau[tid >> 5] = tw;
    if (tid == 0) s_n = 0;
    __syncthreads();
    uint32_t tau = 0xffffffffu;
#pragma unroll
    for (int w = 0; w < kSelWarps; ++w) tau = min(tau, s_wtau[w]);
    uint32_t mine = 0u;
#pragma unroll
    for (int i = 0; i < kSelEPT; ++i)
        if ((valid & (1u << i)) && hw[i] >= tau) mine |= 1u << i;
    // one shared-memory atomic per warp: the warp's candidates go to consecutive slots
    const uint32_t c = __popc(mine);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    uint32_t base = 0u;
    if (lane == 31) base = atomicAdd(reinterpret_cast<uint32_t*>(&s_n), inc);
    base = __shfl_sync(0xffffffffu, base, 31) + inc - c;
#pragma unroll
    for (int i = 0; i < kSelEPT; ++i)
        if (mine & (1u << i)) {
            if (base < static_cast<uint32_t>(kSelCand)) s_cand[base] = key(i);
            ++base;
        }
    __syncthreads();
    const int n_above = s_n;
    __syncthreads();
    if (K > 0 && n_above <= kSelCand) {
        emit_ranked(s_cand, n_above, Kmax, o, tid);
    } else {
        // radix selection of the K-th largest 64-bit key, 8 bits at a time
        if (tid == 0) {
            s_prefix = 0ull;
            s_mask = 0ull;
            s_rem = K;
            s_done = 0;
            s_n = 0;
        }
        __syncthreads();
        for (int shift = 56; shift >= 0 && K > 0 && !s_done; shift -= 8) {
            for (int i = tid; i < 256; i += kSelThreads) s_hist[i] = 0u;
            __syncthreads();
            const uint64_t pre = s_prefix, msk = s_mask;
#pragma unroll
            for (int i = 0; i < kSelEPT; ++i) {
                const uint64_t k = key(i);
                if ((valid & (1u << i)) && (k & msk) == pre) atomicAdd(&s_hist[(k >> shift) & 0xffu], 1u);
            }
            __syncthreads();
            hist_crossing<1>(s_hist, s_rem, tid, s_wsum, &s_bstar, &s_above);
            if (tid == 0) {
                const int d = s_bstar;
                const int rem = s_rem - s_above;
                s_rem = rem;
                s_prefix = pre | (static_cast<uint64_t>(d) << shift);
                s_mask = msk | (0xffull << shift);
                if (shift == 32 && static_cast<int>(s_hist[d]) == rem) s_done = 1;
            }
            __syncthreads();
        }
        // keys are unique (index bits): exactly K keys are >= the K-th one (<= kMaxK)
        const uint64_t kth = s_prefix;
#pragma unroll
        for (int i = 0; i < kSelEPT; ++i) {
            const uint64_t k = key(i);
            if (K > 0 && (valid & (1u << i)) && k >= kth) {
                const int at = atomicAdd(&s_n, 1);
                if (at < kMaxK) s_cand[at] = k;
            }
        }
        __syncthreads();
        emit_ranked(s_cand, min(s_n, kMaxK), Kmax, o, tid);
    }
}

// Level kScores: chunk blockIdx.x of query blockIdx.y.  On the final level the
// last block of a query (ticket) merges the query's chunk lists in the same way;
// the other blocks' lists are visible to it after their fences.
template <bool kScores>
__global__ void __launch_bounds__(kSelThreads, 4) k_topk_select(const __grid_constant__ SelectParams p) {
    __shared__ SelectSmem sm;
    const int q = blockIdx.y, chunk = blockIdx.x;
    const int64_t b = static_cast<int64_t>(chunk) * p.chunk;
    const int64_t rest = p.L - b;
    const int m = static_cast<int>(rest < p.chunk ? rest : p.chunk);
    const float* sc = kScores ? p.scores + static_cast<int64_t>(q) * p.ld + b : nullptr;
    const uint64_t* kr = kScores ? nullptr : p.keys_in + static_cast<int64_t>(q) * p.L + b;
    const SelectOut result{nullptr, p.out_score + static_cast<int64_t>(q) * p.K,
                           p.out_index + static_cast<int64_t>(q) * p.K};
    uint64_t* lists = p.keys_out + static_cast<int64_t>(q) * p.chunks * p.K;
    if (p.tickets && p.chunks == 1) {
        select_block<kScores>(sm, sc, kr, b, m, p.K, result);
        return;
    }
    select_block<kScores>(sm, sc, kr, b, m, p.K, SelectOut{lists + static_cast<int64_t>(chunk) * p.K, nullptr, nullptr});
    if (!p.tickets) return;
    __syncthreads();  // the block's list is written; one fence (cumulative) publishes it
    if (threadIdx.x == 0) {
        __threadfence();
        sm.last = atomicAdd(&p.tickets[q], 1u) == static_cast<uint32_t>(p.chunks - 1);
    }
    __syncthreads();
    if (!sm.last) return;
    __threadfence();
    select_block<false>(sm, nullptr, lists, 0, p.chunks * p.K, p.K, result);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
        cudaGetLastError();
    });
    return fn;
}

// bf16 [rows][D] row-major, tile {64 dims, box_rows}, 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int32_t D, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(D), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(D) * 2};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(kTileK), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

}  // namespace imloc

extern "C" int imloc_retrieve_topk_async(imloc_ctx* ctx, const uint16_t* queries, int32_t n_queries,
                                         const uint16_t* db, int64_t n_db, int32_t dim, int32_t k, float* out_score,
                                         int32_t* out_index, void* stream) {
    using namespace imloc;
    if (!ctx || !queries || !db || !out_score || !out_index) return IMLOC_ERR_INVALID_ARG;
    if (n_queries < 1 || n_db < 1 || n_db > 0x7fffffffLL || dim < 8 || dim % 8 != 0 || k < 1 || k > kMaxK)
        return IMLOC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(queries) | reinterpret_cast<uintptr_t>(db)) & 15u) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    rc = [&]() -> int {
        const int Qg_max = std::min(n_queries, kMaxNq);
        const int64_t ld = (n_db + 3) & ~int64_t{3};  // score rows start 16-byte aligned
        float* scores = static_cast<float*>(ws_alloc(ctx, sizeof(float) * static_cast<size_t>(Qg_max) * ld));
        // selection chunks: small enough to spread few queries over the SMs, while one
        // block can still merge a query's chunk lists
        int chunk0 = kSelectChunk;
        while (chunk0 > 1024 && static_cast<int64_t>(Qg_max) * ((n_db + chunk0 - 1) / chunk0) < 2LL * ctx->sm_count &&
               (n_db + chunk0 / 2 - 1) / (chunk0 / 2) * k <= kSelectChunk)
            chunk0 >>= 1;
        const int chunks0 = static_cast<int>((n_db + chunk0 - 1) / chunk0);
        uint64_t* kbuf[2] = {
            static_cast<uint64_t*>(ws_alloc(ctx, sizeof(uint64_t) * static_cast<size_t>(Qg_max) * chunks0 * k)),
            static_cast<uint64_t*>(ws_alloc(ctx, sizeof(uint64_t) * static_cast<size_t>(Qg_max) * chunks0 * k))};
        uint32_t* tickets = static_cast<uint32_t*>(ws_alloc(ctx, sizeof(uint32_t) * kMaxNq));
        if (!scores || !kbuf[0] || !kbuf[1] || !tickets) return IMLOC_ERR_OOM;
        const int n_tiles = static_cast<int>((n_db + kTileM - 1) / kTileM);
        for (int q0 = 0; q0 < n_queries; q0 += kMaxNq) {
            const int Qg = std::min(kMaxNq, n_queries - q0);
            const int Nq = std::max(16, (Qg + 15) / 16 * 16);
            GemmParams gp;
            memset(&gp, 0, sizeof(gp));
            if (!make_map(&gp.map_db, db, n_db, dim, kTileM) ||
                !make_map(&gp.map_q, queries + static_cast<int64_t>(q0) * dim, Qg, dim, Nq))
                return IMLOC_ERR_CUDA;
            gp.scores = scores;
            gp.ld = ld;
            gp.N = n_db;
            gp.Q = Qg;
            gp.D = dim;
            gp.Nq = Nq;
            const size_t stage = static_cast<size_t>(kTileM) * kTileK * 2 + static_cast<size_t>(Nq) * kTileK * 2;
            // as many stages as ~200 KB of shared memory hold: the bytes in flight hide the DRAM latency
            gp.stages = static_cast<int>(std::min<size_t>(12, std::max<size_t>(2, (200u << 10) / stage)));
            int cols = 32;
            while (cols < 2 * Nq) cols <<= 1;
            gp.tmem_cols = cols;
            gp.n_tiles = n_tiles;
            gp.err = ctx->d_err;
            const size_t smem = 1024 + gp.stages * stage + sizeof(uint64_t) * (2 * gp.stages + 4) + 16;
            IMLOC_CUDA_TRY(cudaFuncSetAttribute(k_retrieve_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(smem)));
            IMLOC_CUDA_TRY(cudaFuncSetAttribute(k_topk_select<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                cudaSharedmemCarveoutMaxShared));
            IMLOC_CUDA_TRY(cudaFuncSetAttribute(k_topk_select<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                cudaSharedmemCarveoutMaxShared));
            const int grid = std::min(n_tiles, ctx->sm_count);
            const size_t vsmem = sizeof(float) * static_cast<size_t>(Qg) * dim;
            if (Qg <= kGemvMaxQ && vsmem <= (160u << 10)) {
                GemvParams vp;
                vp.db = reinterpret_cast<const uint4*>(db);
                vp.q = reinterpret_cast<const uint4*>(queries + static_cast<int64_t>(q0) * dim);
                vp.scores = scores;
                vp.ld = ld;
                vp.N = n_db;
                vp.D8 = dim / 8;
                vp.pad = 0;
                auto kern = Qg == 1 ? k_retrieve_gemv<1> : k_retrieve_gemv<2>;
                IMLOC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(vsmem)));
                int per_sm = 0;
                IMLOC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGemvThreads, vsmem));
                if (per_sm < 1) return IMLOC_ERR_CUDA;
                const int64_t rows_per_block = kGemvThreads / 32;
                const int vgrid = static_cast<int>(
                    std::min<int64_t>(static_cast<int64_t>(per_sm) * ctx->sm_count, (n_db + rows_per_block - 1) / rows_per_block));
                ProfScope prof(ctx, st, "k_retrieve_gemv");
                kern<<<vgrid, kGemvThreads, vsmem, st>>>(vp);
                IMLOC_CUDA_TRY(cudaGetLastError());
                prof.end();
            } else {
                ProfScope prof(ctx, st, "k_retrieve_gemm");
                k_retrieve_gemm<<<grid, kGemmThreads, smem, st>>>(gp);
                IMLOC_CUDA_TRY(cudaGetLastError());
                prof.end();
            }
            // top-K: chunks of up to 4,096 scores, then merge levels; the final level's
            // last block per query writes the result
            SelectParams sp;
            memset(&sp, 0, sizeof(sp));
            sp.scores = scores;
            sp.ld = ld;
            sp.L = n_db;
            sp.K = k;
            sp.chunk = chunk0;
            sp.out_score = out_score + static_cast<int64_t>(q0) * k;
            sp.out_index = out_index + static_cast<int64_t>(q0) * k;
            int chunks = chunks0, cur = 0;
            IMLOC_CUDA_TRY(cudaMemsetAsync(tickets, 0, sizeof(uint32_t) * Qg, st));
            {
                ProfScope prof(ctx, st, "k_topk_select");
                for (;;) {
                    const bool last = static_cast<int64_t>(chunks) * k <= kSelectChunk;
                    sp.chunks = chunks;
                    sp.keys_out = kbuf[cur];
                    sp.tickets = last ? tickets : nullptr;
                    if (sp.scores)
                        k_topk_select<true><<<dim3(chunks, Qg), kSelThreads, 0, st>>>(sp);
                    else
                        k_topk_select<false><<<dim3(chunks, Qg), kSelThreads, 0, st>>>(sp);
                    IMLOC_CUDA_TRY(cudaGetLastError());
                    if (last) break;
                    sp.scores = nullptr;
                    sp.keys_in = kbuf[cur];
                    sp.L = static_cast<int64_t>(chunks) * k;
                    sp.chunk = kSelectChunk;
                    chunks = static_cast<int>((sp.L + kSelectChunk - 1) / kSelectChunk);
                    cur ^= 1;
                }
                prof.end();
            }
        }
        return IMLOC_OK;
    }();
    const int rc2 = end_call(ctx, st);
    return rc != IMLOC_OK ? rc : rc2;
}
