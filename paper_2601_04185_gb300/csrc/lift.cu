// lift.cu -- 2D-2D -> 2D-3D lifting through stored depth maps (ImLoc Sec. 3.3,
// "Query Time Matching and 2D-3D Lifting").
//
// One thread per match: confidence filter (> 0.05 in float32), depth fetch
// (bilinear between the four surrounding pixel centres for query->database
// matches, a single lookup for database->query matches), back-projection
// X_w = R^T (d K^-1 [u v 1]^T - t), then a stable compaction of the valid
// matches into a structure of arrays.  The compaction is single pass: each
// CTA takes the next tile id from an atomic counter, scans its flags with
// warp ballots, publishes its count and looks back over its predecessors'
// published counts/prefixes (decoupled look-back) with a bounded spin.
//
// HBM-bound: per match 20 B of match data, the depth taps (two 32-B sectors
// for a bilinear fetch) and 28 B of output.  Float32 maps may also be stored
// in 4x4-pixel blocks of 64 bytes, so that most bilinear footprints fall in
// one 128-byte line, or in overlapping 8x4-pixel blocks of 128 bytes, so
// that every footprint does.  Views stored as 8-bit log codes
// (the depth codec of Sec. 3.3 "Data Compression") are decoded in the fetch
// through a 256-entry table in shared memory: one byte per tap and a map
// store a quarter of the float32 size (which then mostly stays in L2).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "codec.h"
#include "common.cuh"
#include "ctx.h"

namespace imloc {

struct __align__(16) LiftView {
    const void* depth;    // float32 metres or uint8 log codes (fmt)
    int64_t pitch;
    int32_t W, H;
    int32_t fmt;          // IMLOC_DEPTH_F32 / _LOG8 / _F32_TILE4 / _F32_HALO
    int32_t pad;
    float ifx, ify, cx, cy;
    float Rt[9];  // R^T, row-major
    float C[3];   // camera centre -R^T t
};

struct LiftSeg {
    int64_t begin;
    int32_t view;
    int32_t dir;
    int32_t q_lo, q_hi;  // queries [q_lo, q_hi) whose first match is `begin` (empty range if none)
};
static_assert(sizeof(LiftView) == 96 && sizeof(LiftSeg) == 24, "table entry sizes are part of the scratch budget");

constexpr int kLiftThreads = 256;
static_assert(kLiftThreads == 256, "one decode-table entry per thread");
constexpr int kLiftItems = 4;
constexpr int kLiftTile = kLiftThreads * kLiftItems;
constexpr uint32_t kFlagAggregate = 1u, kFlagPrefix = 2u;
constexpr int kTileSegs = 8;  // segments of one tile staged in shared memory (more: per-match search)

struct LiftParams {
    const float *q_u, *q_v, *db_u, *db_v, *conf;
    int64_t n;
    const LiftSeg* segs;
    const int32_t* tile_seg;  // per tile: (first segment << 4) | segments it touches (0: more than kTileSegs)
    int32_t n_seg;
    int32_t n_tiles;
    const LiftView* views;
    float conf_min;
    uint32_t spin_limit;    // iteration limit of the look-back wait
    float *ox, *oy, *oX, *oY, *oZ, *ow;
    int32_t* osrc;
    int32_t* count;         // total valid (device), may be null
    int64_t* offsets;       // per-query output offsets (device, n_queries+1), may be null
    int32_t tail_q_lo, n_queries;  // queries [tail_q_lo, n_queries] start at n (all take the total)
    unsigned long long* tile_state;  // n_tiles words: (flag << 32) | value
    uint32_t* tile_counter;
    int* err;
    float lut[256];         // log8 code -> metres (code 0 -> 0: no depth)
};

__device__ __forceinline__ bool depth_ok(float d) { return d > 0.0f && d < INFINITY; }

// element offset of pixel (x, y) in the view's map: row-major, or 4x4 blocks
// (the overlapping 8x4 blocks are addressed through halo_offset)
__device__ __forceinline__ int64_t tap_offset(const LiftView& V, int x, int y) {
    if (V.fmt == IMLOC_DEPTH_F32_TILE4)
        return static_cast<int64_t>(y >> 2) * V.pitch + ((x >> 2) << 4) + ((y & 3) << 2) + (x & 3);
    return static_cast<int64_t>(y) * V.pitch + x;
}

// element offset of pixel (x, y) in the overlapping-block layout, read from
// block (x / 7, y / 3): pixels (x + 1, y), (x, y + 1) and (x + 1, y + 1) of
// the same footprint lie in that block at +1, +8 and +9
__device__ __forceinline__ int64_t halo_offset(const LiftView& V, int x, int y) {
    const int bx = x / 7, by = y / 3;
    return static_cast<int64_t>(by) * V.pitch + bx * 32 + (y - 3 * by) * 8 + (x - 7 * bx);
}

// depth tap at element offset `off` of the view's map (metres; 0 = no depth for codes)
__device__ __forceinline__ float depth_tap(const LiftView& V, int64_t off, const float* lut) {
    if (V.fmt == IMLOC_DEPTH_LOG8) return lut[__ldg(static_cast<const uint8_t*>(V.depth) + off)];
    return __ldg(static_cast<const float*>(V.depth) + off);
}

__device__ __forceinline__ int find_segment(const LiftSeg* segs, int n_seg, int64_t j) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].begin <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One tile of kLiftTile matches per CTA, tiles taken in order from an atomic
// counter (every predecessor of a tile has started, so the look-back wait
// ends).  The per-tile latency chain is kept short: the match loads of all
// items are issued right after the tile id is known; warp 0 meanwhile reads
// the tile's segment range from a host-built table and stages the segments
// and their views in shared memory; then every thread issues the depth taps
// of all its items before it uses any of them.
__global__ void __launch_bounds__(kLiftThreads, 4) k_lift(const __grid_constant__ LiftParams p) {
    __shared__ int s_tile;
    __shared__ int s_wcnt[kLiftItems * (kLiftThreads / 32)];
    __shared__ int s_excl;
    __shared__ int s_seg0, s_nseg;
    __shared__ LiftSeg s_seg[kTileSegs];
    __shared__ LiftView s_view[kTileSegs];
    __shared__ float s_lut[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kLiftThreads / 32;
    s_lut[tid] = p.lut[tid];  // kLiftThreads == 256 entries
    if (tid == 0) s_tile = static_cast<int>(atomicAdd(p.tile_counter, 1u));
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = static_cast<int64_t>(tile) * kLiftTile;

    // match data is read once: streaming loads keep L2 for the depth taps
    float mc[kLiftItems], mu[kLiftItems], mv[kLiftItems], vx[kLiftItems], vy[kLiftItems];
#pragma unroll
    for (int k = 0; k < kLiftItems; ++k) {
        const int64_t j = base + k * kLiftThreads + tid;
        if (j < p.n) {
            mc[k] = __ldcs(p.conf + j);
            mu[k] = __ldcs(p.db_u + j);
            mv[k] = __ldcs(p.db_v + j);
            vx[k] = __ldcs(p.q_u + j);
            vy[k] = __ldcs(p.q_v + j);
        } else {
            mc[k] = mu[k] = mv[k] = vx[k] = vy[k] = 0.0f;
        }
    }
    if (warp == 0) {
        const int ts = __ldg(p.tile_seg + tile);
        const int s0 = ts >> 4, ns = ts & 15;
        if (lane < ns) {
            const LiftSeg sg = p.segs[s0 + lane];
            s_seg[lane] = sg;
            s_view[lane] = p.views[sg.view];
        }
        if (lane == 0) { s_seg0 = s0; s_nseg = ns; }
    }
    __syncthreads();
    const int nseg_local = s_nseg, seg0 = s_seg0;

    // segment of every item, its view's taps issued for all items first
    int seg_of[kLiftItems];
    bool want[kLiftItems];
    float t00[kLiftItems], t01[kLiftItems], t10[kLiftItems], t11[kLiftItems];
#pragma unroll
    for (int k = 0; k < kLiftItems; ++k) {
        const int64_t j = base + k * kLiftThreads + tid;
        seg_of[k] = -1;
        want[k] = false;
        t00[k] = t01[k] = t10[k] = t11[k] = 0.0f;
        if (j >= p.n) continue;
        int ls = -1, s;
        if (nseg_local > 0) {
            ls = nseg_local - 1;
            while (ls > 0 && s_seg[ls].begin > j) --ls;
            s = seg0 + ls;
        } else {
            s = find_segment(p.segs, p.n_seg, j);
        }
        seg_of[k] = s;
        if (!(mc[k] > p.conf_min)) continue;
        const LiftSeg& sg = ls >= 0 ? s_seg[ls] : p.segs[s];
        const LiftView& V = ls >= 0 ? s_view[ls] : p.views[sg.view];
        const float u = mu[k], v = mv[k];
        if (sg.dir == 0) {
            const float a = u - 0.5f, b = v - 0.5f;
            if (!((a >= 0.0f) && (a < static_cast<float>(V.W - 1)) && (b >= 0.0f) && (b < static_cast<float>(V.H - 1))))
                continue;
            const int i0 = static_cast<int>(a), j0 = static_cast<int>(b);
            if (V.fmt == IMLOC_DEPTH_F32_HALO) {
                const float* h = static_cast<const float*>(V.depth) + halo_offset(V, i0, j0);
                t00[k] = __ldg(h);
                t01[k] = __ldg(h + 1);
                t10[k] = __ldg(h + 8);
                t11[k] = __ldg(h + 9);
            } else {
                t00[k] = depth_tap(V, tap_offset(V, i0, j0), s_lut);
                t01[k] = depth_tap(V, tap_offset(V, i0 + 1, j0), s_lut);
                t10[k] = depth_tap(V, tap_offset(V, i0, j0 + 1), s_lut);
                t11[k] = depth_tap(V, tap_offset(V, i0 + 1, j0 + 1), s_lut);
            }
        } else {
            if (!((u >= 0.0f) && (u < static_cast<float>(V.W)) && (v >= 0.0f) && (v < static_cast<float>(V.H))))
                continue;
            const int x = static_cast<int>(u), y = static_cast<int>(v);
            t00[k] = V.fmt == IMLOC_DEPTH_F32_HALO ? __ldg(static_cast<const float*>(V.depth) + halo_offset(V, x, y))
                                                   : depth_tap(V, tap_offset(V, x, y), s_lut);
        }
        want[k] = true;
    }

    // depth, validity and back-projection
    float vX[kLiftItems], vY[kLiftItems], vZ[kLiftItems];
    bool ok[kLiftItems];
#pragma unroll
    for (int k = 0; k < kLiftItems; ++k) {
        ok[k] = false;
        vX[k] = vY[k] = vZ[k] = 0.0f;
        if (!want[k]) continue;
        const int s = seg_of[k];
        const int ls = nseg_local > 0 ? s - seg0 : -1;
        const LiftSeg& sg = ls >= 0 ? s_seg[ls] : p.segs[s];
        const LiftView& V = ls >= 0 ? s_view[ls] : p.views[sg.view];
        const float u = mu[k], v = mv[k];
        float d;
        bool good;
        if (sg.dir == 0) {
            const float a = u - 0.5f, b = v - 0.5f;
            const float d00 = t00[k], d01 = t01[k], d10 = t10[k], d11 = t11[k];
            good = depth_ok(d00) && depth_ok(d01) && depth_ok(d10) && depth_ok(d11);
            const float al = a - static_cast<float>(static_cast<int>(a)), be = b - static_cast<float>(static_cast<int>(b));
            d = (1.0f - be) * ((1.0f - al) * d00 + al * d01) + be * ((1.0f - al) * d10 + al * d11);
        } else {
            d = t00[k];
            good = depth_ok(d);
        }
        if (!good) continue;
        const float xc = d * ((u - V.cx) * V.ifx), yc = d * ((v - V.cy) * V.ify), zc = d;
        vX[k] = fmaf(V.Rt[0], xc, fmaf(V.Rt[1], yc, fmaf(V.Rt[2], zc, V.C[0])));
        vY[k] = fmaf(V.Rt[3], xc, fmaf(V.Rt[4], yc, fmaf(V.Rt[5], zc, V.C[1])));
        vZ[k] = fmaf(V.Rt[6], xc, fmaf(V.Rt[7], yc, fmaf(V.Rt[8], zc, V.C[2])));
        ok[k] = true;
    }

    // ---- tile-local scan in input order: item k, then warp, then lane ----
    uint32_t ball[kLiftItems];
#pragma unroll
    for (int k = 0; k < kLiftItems; ++k) {
        ball[k] = __ballot_sync(0xffffffffu, ok[k]);
        if (lane == 0) s_wcnt[k * kWarps + warp] = __popc(ball[k]);
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan over the kLiftItems * kWarps (= 32) warp counts
        const int v = s_wcnt[lane];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        s_wcnt[lane] = incl - v;

        // ---- decoupled look-back over predecessor tiles ----
        int excl = 0;
        if (tile == 0) {
            if (lane == 0)
                atomicExch(&p.tile_state[0], (static_cast<unsigned long long>(kFlagPrefix) << 32) | static_cast<uint32_t>(total));
        } else {
            if (lane == 0)
                atomicExch(&p.tile_state[tile], (static_cast<unsigned long long>(kFlagAggregate) << 32) | static_cast<uint32_t>(total));
            int look = tile - 1;
            uint32_t spins = 0;
            while (true) {
                const int i = look - lane;
                unsigned long long st = (i >= 0) ? *reinterpret_cast<volatile unsigned long long*>(&p.tile_state[i])
                                                 : (static_cast<unsigned long long>(kFlagPrefix) << 32);
                while (__any_sync(0xffffffffu, (st >> 32) == 0u)) {
                    if (++spins > p.spin_limit) {
                        // give up: record the error (before publishing a prefix that rests on it)
                        // and take the unpublished predecessors as empty, so that the kernel ends
                        if (lane == 0) atomicCAS(p.err, 0, kDevTimeoutLookback);
                        __threadfence();
                        if ((st >> 32) == 0u) st = (static_cast<unsigned long long>(kFlagPrefix) << 32);
                        break;
                    }
                    if ((st >> 32) == 0u) st = *reinterpret_cast<volatile unsigned long long*>(&p.tile_state[i]);
                }
                const uint32_t pmask = __ballot_sync(0xffffffffu, (st >> 32) == kFlagPrefix);
                const int val = static_cast<int>(st & 0xffffffffu);
                if (pmask) {
                    const int first = __ffs(pmask) - 1;
                    excl += warp_sum_i(lane <= first ? val : 0);
                    break;
                }
                excl += warp_sum_i(val);
                look -= 32;
            }
            if (lane == 0)
                atomicExch(&p.tile_state[tile],
                           (static_cast<unsigned long long>(kFlagPrefix) << 32) | static_cast<uint32_t>(excl + total));
        }
        if (lane == 0) {
            s_excl = excl;
            if (tile == p.n_tiles - 1) {
                if (p.count) *p.count = excl + total;
                if (p.offsets)
                    for (int q = p.tail_q_lo; q <= p.n_queries; ++q) p.offsets[q] = excl + total;
            }
        }
    }
    __syncthreads();

    const uint32_t lt = (1u << lane) - 1u;
    const int excl = s_excl;
#pragma unroll
    for (int k = 0; k < kLiftItems; ++k) {
        const int pos = excl + s_wcnt[k * kWarps + warp] + __popc(ball[k] & lt);
        const int64_t j = base + k * kLiftThreads + tid;
        if (seg_of[k] >= 0 && p.offsets) {
            const LiftSeg& sg = p.segs[seg_of[k]];
            if (sg.begin == j)
                for (int q = sg.q_lo; q < sg.q_hi; ++q) p.offsets[q] = pos;
        }
        if (!ok[k]) continue;
        p.ox[pos] = vx[k];
        p.oy[pos] = vy[k];
        p.oX[pos] = vX[k];
        p.oY[pos] = vY[k];
        p.oZ[pos] = vZ[k];
        p.ow[pos] = mc[k];
        p.osrc[pos] = static_cast<int32_t>(j);
    }
}

// ---- host side ---------------------------------------------------------------

// Argument checks shared by every lift entry point.
static int check_lift_args(const imloc_view* views, int32_t n_views, const imloc_matches* m, const imloc_corr* out) {
    if (!views || n_views <= 0 || !m || !out) return IMLOC_ERR_INVALID_ARG;
    if (m->n < 0 || m->n >= (int64_t(1) << 31)) return IMLOC_ERR_INVALID_ARG;
    if (out->capacity < m->n) return IMLOC_ERR_CAPACITY;
    if (m->n > 0) {
        if (!m->q_u || !m->q_v || !m->db_u || !m->db_v || !m->conf || !m->segments || m->n_segments <= 0)
            return IMLOC_ERR_INVALID_ARG;
        if (!out->x || !out->y || !out->X || !out->Y || !out->Z || !out->w || !out->src) return IMLOC_ERR_INVALID_ARG;
        if (m->segments[0].begin != 0) return IMLOC_ERR_INVALID_ARG;
    }
    for (int s = 0; s < m->n_segments; ++s) {
        const imloc_segment& sg = m->segments[s];
        if (sg.view < 0 || sg.view >= n_views || (sg.direction != 0 && sg.direction != 1)) return IMLOC_ERR_INVALID_ARG;
        if (s > 0 && sg.begin < m->segments[s - 1].begin) return IMLOC_ERR_INVALID_ARG;
        if (sg.begin > m->n) return IMLOC_ERR_INVALID_ARG;
    }
    for (int v = 0; v < n_views; ++v) {
        const imloc_view& V = views[v];
        if (!V.depth || V.width < 2 || V.height < 2 || V.pitch < V.width) return IMLOC_ERR_INVALID_ARG;
        if (!(V.cam.fx != 0.0f) || !(V.cam.fy != 0.0f)) return IMLOC_ERR_INVALID_ARG;
        if (V.depth_format != IMLOC_DEPTH_F32 && V.depth_format != IMLOC_DEPTH_LOG8 &&
            V.depth_format != IMLOC_DEPTH_F32_TILE4 && V.depth_format != IMLOC_DEPTH_F32_HALO)
            return IMLOC_ERR_INVALID_ARG;
        if (V.depth_format == IMLOC_DEPTH_F32_TILE4 && (V.pitch % 16 != 0 || V.pitch < 16 * ((V.width + 3) / 4)))
            return IMLOC_ERR_INVALID_ARG;
        if (V.depth_format == IMLOC_DEPTH_F32_HALO && (V.pitch % 32 != 0 || V.pitch < 32 * ((V.width - 1) / 7 + 1)))
            return IMLOC_ERR_INVALID_ARG;
    }
    return IMLOC_OK;
}

// Device-side view entry: inverse focal lengths, R^T and the camera centre in float32.
static void fill_view(const imloc_view& V, LiftView& L) {
    L.depth = V.depth;
    L.pitch = V.pitch;
    L.W = V.width;
    L.H = V.height;
    L.fmt = V.depth_format;
    L.pad = 0;
    L.ifx = static_cast<float>(1.0 / static_cast<double>(V.cam.fx));
    L.ify = static_cast<float>(1.0 / static_cast<double>(V.cam.fy));
    L.cx = V.cam.cx;
    L.cy = V.cam.cy;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) L.Rt[3 * r + c] = static_cast<float>(V.pose.R[3 * c + r]);
    for (int r = 0; r < 3; ++r) {
        double cr = 0.0;
        for (int c = 0; c < 3; ++c) cr -= V.pose.R[3 * c + r] * V.pose.t[c];
        L.C[r] = static_cast<float>(cr);
    }
}

// Per tile: its first segment and how many segments it touches (segments
// sorted by begin, non-empty, covering [0, n)).
static void fill_tile_segments(const LiftSeg* segs, int n_seg, int64_t n, int n_tiles, int32_t* tile_seg) {
    int s = 0;
    for (int t = 0; t < n_tiles; ++t) {
        const int64_t b = static_cast<int64_t>(t) * kLiftTile;
        const int64_t e = std::min(b + kLiftTile, n) - 1;
        while (s + 1 < n_seg && segs[s + 1].begin <= b) ++s;
        int s1 = s;
        while (s1 + 1 < n_seg && segs[s1 + 1].begin <= e) ++s1;
        const int ns = s1 - s + 1;
        tile_seg[t] = (s << 4) | (ns <= kTileSegs ? ns : 0);
    }
}

// Test hook state: the look-back limit of the next lift and the tiles it skips.
struct LiftTestHooks {
    uint32_t spin_limit = kSpinLimit;
    int skip_tiles = 0;
};

static int lift_launch(imloc_ctx* ctx, int32_t n_queries, const int64_t* query_begin, const imloc_view* views,
                       int32_t n_views, const imloc_matches* m, imloc_corr* out, int64_t* d_offsets,
                       cudaStream_t stream, const LiftTestHooks& hooks) {
    if (n_queries <= 0 || !query_begin) return IMLOC_ERR_INVALID_ARG;
    int rc = check_lift_args(views, n_views, m, out);
    if (rc != IMLOC_OK) return rc;
    if (query_begin[0] != 0 || query_begin[n_queries] != m->n) return IMLOC_ERR_INVALID_ARG;
    for (int q = 0; q < n_queries; ++q)
        if (query_begin[q + 1] < query_begin[q]) return IMLOC_ERR_INVALID_ARG;

    // Device segment table: non-empty segments only; every query must begin at
    // the start of one of them, or at n (then it is empty and takes the total).
    std::vector<LiftSeg> segs;
    int qi = 0;
    for (int s = 0; s < (m->n > 0 ? m->n_segments : 0); ++s) {
        const int64_t b = m->segments[s].begin;
        const int64_t e = (s + 1 < m->n_segments) ? m->segments[s + 1].begin : m->n;
        if (e <= b) continue;
        LiftSeg L;
        L.begin = b;
        L.view = m->segments[s].view;
        L.dir = m->segments[s].direction;
        if (qi < n_queries && query_begin[qi] < b) return IMLOC_ERR_INVALID_ARG;  // begins inside a segment
        L.q_lo = qi;
        while (qi < n_queries && query_begin[qi] == b) ++qi;
        L.q_hi = qi;
        segs.push_back(L);
    }
    for (int q = qi; q < n_queries; ++q)
        if (query_begin[q] != m->n) return IMLOC_ERR_INVALID_ARG;
    const int tail_q_lo = qi;

    const int64_t n = m->n;
    const int n_tiles = static_cast<int>((n + kLiftTile - 1) / kLiftTile);
    if (n == 0) {
        if (out->count) IMLOC_CUDA_TRY(cudaMemsetAsync(out->count, 0, sizeof(int32_t), stream));
        if (d_offsets) IMLOC_CUDA_TRY(cudaMemsetAsync(d_offsets, 0, sizeof(int64_t) * (n_queries + 1), stream));
        return IMLOC_OK;
    }
    if (hooks.skip_tiles >= n_tiles) return IMLOC_ERR_INVALID_ARG;
    const size_t seg_bytes = sizeof(LiftSeg) * segs.size(), view_bytes = sizeof(LiftView) * n_views;
    const size_t view_off = align_up(seg_bytes, 256);
    const size_t ts_off = view_off + align_up(view_bytes, 256);
    const size_t total = ts_off + sizeof(int32_t) * n_tiles;
    char* h = static_cast<char*>(staging_alloc(ctx, total));
    char* d = static_cast<char*>(ws_alloc(ctx, total));
    if (!h || !d) return IMLOC_ERR_OOM;
    memcpy(h, segs.data(), seg_bytes);
    LiftView* hv = reinterpret_cast<LiftView*>(h + view_off);
    for (int v = 0; v < n_views; ++v) fill_view(views[v], hv[v]);
    fill_tile_segments(segs.data(), static_cast<int>(segs.size()), n, n_tiles, reinterpret_cast<int32_t*>(h + ts_off));
    rc = upload(ctx, d, h, total, stream);
    if (rc != IMLOC_OK) return rc;

    // scan scratch: word 0 = tile counter, words 1..n_tiles = tile states
    unsigned long long* state = static_cast<unsigned long long*>(ws_alloc(ctx, sizeof(unsigned long long) * (n_tiles + 1)));
    if (!state) return IMLOC_ERR_OOM;
    IMLOC_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(unsigned long long) * (n_tiles + 1), stream));
    if (hooks.skip_tiles > 0)  // test hook: the first tiles are never taken (their states stay unpublished)
        IMLOC_CUDA_TRY(cudaMemsetAsync(state, hooks.skip_tiles, 1, stream));

    LiftParams p;
    p.q_u = m->q_u; p.q_v = m->q_v; p.db_u = m->db_u; p.db_v = m->db_v; p.conf = m->conf;
    p.n = n;
    p.segs = reinterpret_cast<const LiftSeg*>(d);
    p.tile_seg = reinterpret_cast<const int32_t*>(d + ts_off);
    p.n_seg = static_cast<int32_t>(segs.size());
    p.n_tiles = n_tiles;
    p.views = reinterpret_cast<const LiftView*>(d + view_off);
    p.conf_min = 0.05f;
    p.spin_limit = hooks.spin_limit;
    p.ox = out->x; p.oy = out->y; p.oX = out->X; p.oY = out->Y; p.oZ = out->Z; p.ow = out->w;
    p.osrc = out->src;
    p.count = out->count;
    p.offsets = d_offsets;
    p.tail_q_lo = tail_q_lo;
    p.n_queries = n_queries;
    p.tile_state = state + 1;
    p.tile_counter = reinterpret_cast<uint32_t*>(state);
    p.err = ctx->d_err;
    log8_decode_table(p.lut);
    ProfScope prof(ctx, stream, "k_lift");
    k_lift<<<n_tiles - hooks.skip_tiles, kLiftThreads, 0, stream>>>(p);
    IMLOC_CUDA_TRY(cudaGetLastError());
    prof.end();
    return IMLOC_OK;
}

int lift_impl(imloc_ctx* ctx, int32_t n_queries, const int64_t* query_begin, const imloc_view* views,
              int32_t n_views, const imloc_matches* m, imloc_corr* out, int64_t* d_offsets, cudaStream_t stream) {
    return lift_launch(ctx, n_queries, query_begin, views, n_views, m, out, d_offsets, stream, LiftTestHooks());
}

}  // namespace imloc

extern "C" {

int imloc_lift_async(imloc_ctx* ctx, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                     imloc_corr* out, void* stream) {
    if (!ctx || !m) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = imloc::begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    const int64_t qb[2] = {0, m->n};
    rc = imloc::lift_impl(ctx, 1, qb, views, n_views, m, out, nullptr, st);
    int rc2 = imloc::end_call(ctx, st);
    return rc != IMLOC_OK ? rc : rc2;
}

int imloc_lift_batch_async(imloc_ctx* ctx, int32_t n_queries, const int64_t* query_begin, const imloc_view* views,
                           int32_t n_views, const imloc_matches* m, imloc_corr* out, int64_t* d_offsets,
                           void* stream) {
    if (!ctx || !m) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = imloc::begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    rc = imloc::lift_impl(ctx, n_queries, query_begin, views, n_views, m, out, d_offsets, st);
    int rc2 = imloc::end_call(ctx, st);
    return rc != IMLOC_OK ? rc : rc2;
}

int imloc_testing_lift_stalled(imloc_ctx* ctx, const imloc_view* views, int32_t n_views, const imloc_matches* m,
                               imloc_corr* out, int32_t skip_tiles, uint32_t spin_limit, void* stream) {
    if (!ctx || !m || skip_tiles < 1 || skip_tiles > 255 || spin_limit < 1) return IMLOC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    IMLOC_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = imloc::begin_call(ctx, st);
    if (rc != IMLOC_OK) return rc;
    const int64_t qb[2] = {0, m->n};
    imloc::LiftTestHooks hooks;
    hooks.skip_tiles = skip_tiles;
    hooks.spin_limit = spin_limit;
    rc = imloc::lift_launch(ctx, 1, qb, views, n_views, m, out, nullptr, st, hooks);
    int rc2 = imloc::end_call(ctx, st);
    return rc != IMLOC_OK ? rc : rc2;
}

}  // extern "C"

// ============================================================================
// Allocation-free lift.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool or budget that it does not own, hosts that reserve all device
// memory up front for other components, and callers that must not create a
// context (imloc_create allocates a workspace).  imloc_lift_noalloc_async
// gives them the lift without any allocation: its scratch (the scan state of
// the stable compaction, the view / segment / tile tables and an error word)
// lives in the fixed-size file-scope array below, which every GPU that loads
// this library holds until the process exits.
// ============================================================================
namespace imloc {

constexpr int kNoAllocMaxTiles = 8192;  // 8192 tiles x 1024 matches = 8,388,608 matches per call
constexpr int kNoAllocMaxViews = 256;
constexpr int kNoAllocMaxSegments = 1024;
constexpr size_t noalloc_round256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kNoAllocScanBytes = noalloc_round256(sizeof(unsigned long long) * (kNoAllocMaxTiles + 1));
constexpr size_t kNoAllocSegBytes = noalloc_round256(sizeof(LiftSeg) * kNoAllocMaxSegments);
constexpr size_t kNoAllocViewBytes = noalloc_round256(sizeof(LiftView) * kNoAllocMaxViews);
constexpr size_t kNoAllocTileBytes = noalloc_round256(sizeof(int32_t) * kNoAllocMaxTiles);
constexpr size_t kNoAllocScratchBytes = kNoAllocScanBytes + kNoAllocSegBytes + kNoAllocViewBytes + kNoAllocTileBytes + 256;
// the size the header documents: 65,792 + 24,576 + 24,576 + 32,768 + 256
static_assert(kNoAllocScratchBytes == 147968, "documented scratch size of imloc_lift_noalloc_async");

// In host code this name is only a stand-in for the device array: its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_lift_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_addr[kNoAllocMaxDevices];

// After the lift: a look-back that gave up replaces the count by IMLOC_ERR_TIMEOUT.
__global__ void k_lift_noalloc_status(const int* err, int32_t* count) {
    if (*err != 0) *count = IMLOC_ERR_TIMEOUT;
}

}  // namespace imloc

extern "C" int imloc_lift_noalloc_async(const imloc_view* views, int32_t n_views, const imloc_matches* m,
                                        imloc_corr* out, void* stream) {
    using namespace imloc;
    int rc = check_lift_args(views, n_views, m, out);
    if (rc != IMLOC_OK) return rc;
    // fixed limits of the static scratch
    if (m->n > static_cast<int64_t>(kNoAllocMaxTiles) * kLiftTile) return IMLOC_ERR_INVALID_ARG;
    if (n_views > kNoAllocMaxViews || m->n_segments > kNoAllocMaxSegments) return IMLOC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the tables are copied from this call's host stack: a graph captured from
    // this call would keep pointers into a stack frame that is gone
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    IMLOC_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return IMLOC_ERR_INVALID_ARG;

    // device address of the scratch array, looked up once per device
    int dev = 0;
    IMLOC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return IMLOC_ERR_INVALID_ARG;
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* ptr = nullptr;
            IMLOC_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_lift_noalloc_scratch));
            g_noalloc_addr[dev] = static_cast<unsigned char*>(ptr);
        }
        base = g_noalloc_addr[dev];
    }
    unsigned long long* scan = reinterpret_cast<unsigned long long*>(base);
    LiftSeg* d_segs = reinterpret_cast<LiftSeg*>(base + kNoAllocScanBytes);
    LiftView* d_views = reinterpret_cast<LiftView*>(base + kNoAllocScanBytes + kNoAllocSegBytes);
    int32_t* d_tiles = reinterpret_cast<int32_t*>(base + kNoAllocScanBytes + kNoAllocSegBytes + kNoAllocViewBytes);
    int* d_err = reinterpret_cast<int*>(base + kNoAllocScanBytes + kNoAllocSegBytes + kNoAllocViewBytes +
                                        kNoAllocTileBytes);

    if (m->n == 0) {
        if (out->count) IMLOC_CUDA_TRY(cudaMemsetAsync(out->count, 0, sizeof(int32_t), st));
        return IMLOC_OK;
    }
    // tables in fixed-size host arrays (no heap), copied into the scratch
    LiftSeg segs[kNoAllocMaxSegments];
    LiftView lv[kNoAllocMaxViews];
    int32_t tile_seg[kNoAllocMaxTiles];
    int n_seg = 0;
    for (int s = 0; s < m->n_segments; ++s) {
        const int64_t b = m->segments[s].begin;
        const int64_t e = (s + 1 < m->n_segments) ? m->segments[s + 1].begin : m->n;
        if (e <= b) continue;
        LiftSeg& L = segs[n_seg++];
        L.begin = b;
        L.view = m->segments[s].view;
        L.dir = m->segments[s].direction;
        L.q_lo = L.q_hi = 0;
    }
    for (int v = 0; v < n_views; ++v) fill_view(views[v], lv[v]);
    const int n_tiles = static_cast<int>((m->n + kLiftTile - 1) / kLiftTile);
    fill_tile_segments(segs, n_seg, m->n, n_tiles, tile_seg);
    // the array keeps the previous call's contents: clear the scan state and the error word
    IMLOC_CUDA_TRY(cudaMemcpyAsync(d_segs, segs, sizeof(LiftSeg) * n_seg, cudaMemcpyHostToDevice, st));
    IMLOC_CUDA_TRY(cudaMemcpyAsync(d_views, lv, sizeof(LiftView) * n_views, cudaMemcpyHostToDevice, st));
    IMLOC_CUDA_TRY(cudaMemcpyAsync(d_tiles, tile_seg, sizeof(int32_t) * n_tiles, cudaMemcpyHostToDevice, st));
    IMLOC_CUDA_TRY(cudaMemsetAsync(scan, 0, sizeof(unsigned long long) * (n_tiles + 1), st));
    IMLOC_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));

    LiftParams p;
    p.q_u = m->q_u; p.q_v = m->q_v; p.db_u = m->db_u; p.db_v = m->db_v; p.conf = m->conf;
    p.n = m->n;
    p.segs = d_segs;
    p.tile_seg = d_tiles;
    p.n_seg = n_seg;
    p.n_tiles = n_tiles;
    p.views = d_views;
    p.conf_min = 0.05f;
    p.spin_limit = kSpinLimit;
    p.ox = out->x; p.oy = out->y; p.oX = out->X; p.oY = out->Y; p.oZ = out->Z; p.ow = out->w;
    p.osrc = out->src;
    p.count = out->count;
    p.offsets = nullptr;
    p.tail_q_lo = 1;
    p.n_queries = 0;
    p.tile_state = scan + 1;
    p.tile_counter = reinterpret_cast<uint32_t*>(scan);
    p.err = d_err;
    log8_decode_table(p.lut);
    k_lift<<<n_tiles, kLiftThreads, 0, st>>>(p);
    IMLOC_CUDA_TRY(cudaGetLastError());
    if (out->count) {
        k_lift_noalloc_status<<<1, 1, 0, st>>>(d_err, out->count);
        IMLOC_CUDA_TRY(cudaGetLastError());
    }
    return IMLOC_OK;
}
