// triangulate.cu -- dense triangulation of a mapping depth map (ImLoc
// Sec. 3.3 "Depth Estimation by Dense Matching"): with all poses known, each
// match of a reference pixel fixes its depth up to one degree of freedom;
// the hypothesis with the most inliers at a 2-degree angular threshold wins
// and is refined on the confidence-weighted squared angular errors of its
// inliers; depths with more than 3 inliers are kept.
//
// One CTA per 256 reference pixels, FP32: selection per pixel, then the
// kept pixels compacted in shared memory and refined one per thread.
// Per-source ray matrices
// M_s = R_s^T K_s^-1 and centres live in the kernel parameters.  The
// closest-approach depth is evaluated with cross products (no cancellation
// in |d0 x d1|^2 for small ray angles); the inlier test compares
// |a x d|^2 < tan^2(thr) (a.d)^2, a.d > 0 (no trigonometry); the refinement
// is Gauss-Newton on the angular error vectors (the logarithm map of the
// direction a/|a| around the match's ray, length = the angle, smooth through
// zero), with the step halved until the weighted sum of squared angles
// drops.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace imloc {

namespace {

struct TriParams {
    const float *u, *v, *conf;
    int64_t stride;
    float* depth;
    uint8_t* inliers;
    int32_t W, H, S;
    float conf_min, tan2_thr;
    int32_t keep_more_than, refine_iters;
    float M0[9], C0[3];
    float M[IMLOC_TRIANGULATE_MAX_SOURCES][9];
    float W0[IMLOC_TRIANGULATE_MAX_SOURCES][3];  // C0 - C_s
};

__device__ __forceinline__ void cross(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot(const float a[3], const float b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// atan(x) / x and (d/dx (atan(x) / x)) / x for x^2 = x2 <= 0.04, by their
// Taylor series about 0 (alternating; the first omitted terms, x^12 / 13
// and 12 x^10 / 13, are below 3e-10 and 1e-7 of the sums at x = 0.2)
__device__ __forceinline__ float atan_over_x(float x2) {
    return fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 11.0f, 1.0f / 9.0f), -1.0f / 7.0f), 0.2f),
                         -1.0f / 3.0f), 1.0f);
}
__device__ __forceinline__ float datan_over_x_dx_over_x(float x2) {
    return fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -10.0f / 11.0f, 8.0f / 9.0f), -6.0f / 7.0f), 0.8f), -2.0f / 3.0f);
}

// angle between a and d: atan2(|a x d^|, a.d^) (rho = |a x d^|, p3 = a.d^),
// by the series when the angle is below atan(0.2) = 11.3 degrees
__device__ __forceinline__ float ray_angle(float rho, float p3) {
    if (p3 > 0.0f && rho <= 0.2f * p3) {
        const float x = __fdividef(rho, p3);  // 2-ulp division: well below the angle's use as a cost
        return x * atan_over_x(x * x);
    }
    return atan2f(rho, p3);
}

// the error vector's value and Jacobian along z (da/dz = q): the error vector
// r = theta / rho (p1, p2) with p = (a.e1, a.e2, a.d^), rho = |(p1, p2)|,
// theta = atan2(rho, p3); writes r and dr/dz (zero when a points exactly
// away from d^, where no error vector is defined)
__device__ __forceinline__ void angle_residual(const float a[3], const float q[3], const float dh[3], const float e1[3],
                                               const float e2[3], float r[2], float J[2]) {
    const float p1 = dot(a, e1), p2 = dot(a, e2), p3 = dot(a, dh);
    const float q1 = dot(q, e1), q2 = dot(q, e2), q3 = dot(q, dh);
    const float rho2 = p1 * p1 + p2 * p2;
    const float rho = sqrtf(rho2);
    float f, f_rho, f_p3;
    if (p3 > 0.0f && rho <= 0.2f * p3) {
        // f = atan(x) / (x p3) with x = rho / p3: series in x^2
        // (2-ulp divisions: the Jacobian steers the iteration, the cost test decides it)
        const float ip3 = __fdividef(1.0f, p3);
        const float x2 = rho2 * (ip3 * ip3);
        f = atan_over_x(x2) * ip3;
        f_rho = rho * datan_over_x_dx_over_x(x2) * (ip3 * ip3 * ip3);
        f_p3 = -__fdividef(ip3 * ip3, 1.0f + x2);
    } else if (rho > 0.0f) {
        const float th = atan2f(rho, p3);
        const float den = rho2 + p3 * p3;
        f = th / rho;
        f_rho = (rho * p3 / den - th) / rho2;
        f_p3 = -1.0f / den;
    } else {
        f = f_rho = f_p3 = 0.0f;
    }
    const float drho = rho > 0.0f ? __fdividef(p1 * q1 + p2 * q2, rho) : 0.0f;
    const float df = f_rho * drho + f_p3 * q3;
    r[0] = f * p1;
    r[1] = f * p2;
    J[0] = df * p1 + f * q1;
    J[1] = df * p2 + f * q2;
}

// The rays of pixel px: its own (d0) and one per source match (ds), the
// match confidences and the mask of matches with conf >= conf_min.
template <int MAXS>
__device__ __forceinline__ void pixel_rays(const TriParams& p, int64_t px, float d0[3], float ds[MAXS][3], float cf[MAXS],
                                           uint32_t& used) {
    const int j = static_cast<int>(px / p.W), i = static_cast<int>(px - static_cast<int64_t>(j) * p.W);
    const float x = static_cast<float>(i) + 0.5f, y = static_cast<float>(j) + 0.5f;
#pragma unroll
    for (int r = 0; r < 3; ++r) d0[r] = fmaf(p.M0[3 * r], x, fmaf(p.M0[3 * r + 1], y, p.M0[3 * r + 2]));
    used = 0u;
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
        cf[s] = 0.f;
        ds[s][0] = ds[s][1] = ds[s][2] = 0.f;
        if (s < p.S) {
            const float us = __ldg(p.u + s * p.stride + px), vs = __ldg(p.v + s * p.stride + px);
            cf[s] = __ldg(p.conf + s * p.stride + px);
            if (cf[s] >= p.conf_min) used |= 1u << s;
#pragma unroll
            for (int r = 0; r < 3; ++r) ds[s][r] = fmaf(p.M[s][3 * r], us, fmaf(p.M[s][3 * r + 1], vs, p.M[s][3 * r + 2]));
        }
    }
}

// One CTA per 256 pixels, in two phases.  Selection (every pixel): the
// hypotheses and their inlier tests, branch-free; pixels without a kept
// depth are written at once, kept ones go to a queue in shared memory
// (pixel, winning depth, inlier mask).  Refinement: thread t refines queue
// entry t (its rays recomputed from the match planes, now in L1/L2), so that
// the warps of this phase hold kept pixels only, instead of the ~60 % of
// lanes a per-pixel loop would keep busy.  Results do not depend on the
// queue order.
template <int MAXS>
__global__ void __launch_bounds__(256, MAXS <= 8 ? 3 : 1) k_triangulate(const __grid_constant__ TriParams p) {
    __shared__ int s_nq;
    __shared__ int s_pix[256];
    __shared__ float s_z[256];
    __shared__ uint32_t s_set[256];
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t n = static_cast<int64_t>(p.W) * p.H;
    const int64_t px = static_cast<int64_t>(blockIdx.x) * 256 + tid;
    if (tid == 0) s_nq = 0;
    __syncthreads();
    bool kept = false;
    float best_z = 0.f;
    uint32_t best_set = 0u;
    if (px < n) {
        float d0[3], ds[MAXS][3], cf[MAXS];
        uint32_t used;
        pixel_rays<MAXS>(p, px, d0, ds, cf, used);
        // hypotheses: closest approach of the reference ray to each used match's ray;
        // every loop runs over all sources with predicated updates (pixels of a
        // warp use different matches: branches would serialise them)
        int best_n = 0, best_s = -1;
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
            float nrm[3], wx[3];
            cross(d0, ds[s], nrm);
            cross(p.W0[s], ds[s], wx);
            const float nn = dot(nrm, nrm);
            const float z = -dot(wx, nrm) / nn;
            const bool valid = ((used >> s) & 1u) && nn > 1e-12f * dot(d0, d0) * dot(ds[s], ds[s]) && z > 0.f;
            int cnt = 0;
            uint32_t set = 0u;
#pragma unroll
            for (int k = 0; k < MAXS; ++k) {
                float a[3], c[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) a[r] = fmaf(z, d0[r], p.W0[k][r]);
                cross(a, ds[k], c);
                const float ad = dot(a, ds[k]);
                const bool in = ((used >> k) & 1u) && ad > 0.f && dot(c, c) < p.tan2_thr * ad * ad;
                cnt += in ? 1 : 0;
                set |= in ? (1u << k) : 0u;
            }
            const bool take = valid && cnt > best_n;
            best_n = take ? cnt : best_n;
            best_s = take ? s : best_s;
            best_z = take ? z : best_z;
            best_set = take ? set : best_set;
        }
        kept = best_s >= 0 && best_n > p.keep_more_than;
        if (!kept) p.depth[px] = 0.f;
        if (p.inliers) p.inliers[px] = static_cast<uint8_t>(best_n);
    }
    // queue the kept pixels of the block (one shared atomic per warp)
    const uint32_t bal = __ballot_sync(0xffffffffu, kept);
    int at = 0;
    if (lane == 0 && bal) at = atomicAdd(&s_nq, __popc(bal));
    at = __shfl_sync(0xffffffffu, at, 0) + __popc(bal & ((1u << lane) - 1u));
    if (kept) {
        s_pix[at] = tid;
        s_z[at] = best_z;
        s_set[at] = best_set;
    }
    __syncthreads();
    if (tid >= s_nq) return;
    // refinement of queue entry tid: Gauss-Newton on the angular error vectors
    // of the winner's inliers, weight 0 for the others
    const int64_t qx = static_cast<int64_t>(blockIdx.x) * 256 + s_pix[tid];
    const uint32_t set = s_set[tid];
    float d0[3], ds[MAXS][3], cf[MAXS];
    uint32_t used;
    pixel_rays<MAXS>(p, qx, d0, ds, cf, used);
    float wk[MAXS], e1[MAXS][3], e2[MAXS][3], dh[MAXS][3];
#pragma unroll
    for (int k = 0; k < MAXS; ++k) {
        wk[k] = ((set >> k) & 1u) ? cf[k] : 0.f;
        // unit ray and an orthonormal basis of the plane across it
        const float inv = rsqrtf(fmaxf(dot(ds[k], ds[k]), 1e-30f));
        dh[k][0] = ds[k][0] * inv; dh[k][1] = ds[k][1] * inv; dh[k][2] = ds[k][2] * inv;
        const bool xs = fabsf(dh[k][0]) < 0.9f;
        const float hx[3] = {xs ? 1.f : 0.f, xs ? 0.f : 1.f, 0.f};
        cross(dh[k], hx, e1[k]);
        const float i1 = rsqrtf(fmaxf(dot(e1[k], e1[k]), 1e-30f));
        e1[k][0] *= i1; e1[k][1] *= i1; e1[k][2] *= i1;
        cross(dh[k], e1[k], e2[k]);
    }
    // weighted sum of squared angles over the winner's inliers (sources of
    // weight 0 add nothing and are skipped)
    auto cost = [&](float zz) {
        float e = 0.f;
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
            if (!(wk[k] > 0.f)) continue;
            float a[3], c[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) a[r] = fmaf(zz, d0[r], p.W0[k][r]);
            cross(a, dh[k], c);
            const float th = ray_angle(sqrtf(dot(c, c)), dot(a, dh[k]));
            e = fmaf(wk[k] * th, th, e);
        }
        return e;
    };
    float z = s_z[tid];
    float e = cost(z);
    for (int it = 0; it < p.refine_iters; ++it) {
        float g = 0.f, h = 0.f;
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
            if (!(wk[k] > 0.f)) continue;
            float a[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) a[r] = fmaf(z, d0[r], p.W0[k][r]);
            float rv[2], J[2];
            angle_residual(a, d0, dh[k], e1[k], e2[k], rv, J);
            g = fmaf(wk[k], fmaf(rv[0], J[0], rv[1] * J[1]), g);
            h = fmaf(wk[k], fmaf(J[0], J[0], J[1] * J[1]), h);
        }
        if (!(h > 0.f)) break;
        // steps below ~8 float ulps of z cannot be resolved: that is convergence
        const float tiny = 1e-6f * z;
        float step = -g / h;
        bool accepted = false;
        for (int half = 0; half < 8 && fabsf(step) > tiny; ++half, step *= 0.5f) {
            const float zn = z + step;
            if (!(zn > 0.f)) continue;
            const float en = cost(zn);
            if (en < e) {
                z = zn;
                e = en;
                accepted = true;
                break;
            }
        }
        if (!accepted || fabsf(step) <= tiny) break;
    }
    p.depth[qx] = z;
}

void ray_matrix(const imloc_camera& K, const imloc_pose& P, float M[9], float C[3]) {
    // M = R^T K^-1 (K^-1 = [[1/fx, 0, -cx/fx], [0, 1/fy, -cy/fy], [0, 0, 1]]), C = -R^T t
    const double ki[9] = {1.0 / K.fx, 0.0, -K.cx / K.fx, 0.0, 1.0 / K.fy, -K.cy / K.fy, 0.0, 0.0, 1.0};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += P.R[3 * k + r] * ki[3 * k + c];
            M[3 * r + c] = static_cast<float>(acc);
        }
        double cr = 0.0;
        for (int k = 0; k < 3; ++k) cr -= P.R[3 * k + r] * P.t[k];
        C[r] = static_cast<float>(cr);
    }
}

}  // namespace

}  // namespace imloc

extern "C" {

void imloc_triangulate_default_opts(imloc_triangulate_opts* out) {
    if (!out) return;
    out->angle_deg = 2.0f;       // Sec. 3.3: angular error threshold of 2 degrees
    out->conf_min = 0.05f;       // Sec. 3.3: matches with confidence >= 0.05
    out->keep_more_than = 3;     // Sec. 3.3: keep depths with more than 3 inliers
    out->refine_iters = 20;
}

int imloc_triangulate_depth_async(const imloc_camera* ref_cam, const imloc_pose* ref_pose, int32_t width,
                                  int32_t height, const imloc_camera* src_cams, const imloc_pose* src_poses,
                                  int32_t n_src, const float* u, const float* v, const float* conf,
                                  int64_t plane_stride, const imloc_triangulate_opts* opts, float* depth_out,
                                  uint8_t* inliers_out, void* stream) {
    using namespace imloc;
    if (!ref_cam || !ref_pose || !src_cams || !src_poses || !u || !v || !conf || !opts || !depth_out)
        return IMLOC_ERR_INVALID_ARG;
    if (width < 1 || height < 1 || n_src < 1 || n_src > IMLOC_TRIANGULATE_MAX_SOURCES) return IMLOC_ERR_INVALID_ARG;
    if (plane_stride < static_cast<int64_t>(width) * height) return IMLOC_ERR_INVALID_ARG;
    if (!(ref_cam->fx != 0.f) || !(ref_cam->fy != 0.f)) return IMLOC_ERR_INVALID_ARG;
    for (int s = 0; s < n_src; ++s)
        if (!(src_cams[s].fx != 0.f) || !(src_cams[s].fy != 0.f)) return IMLOC_ERR_INVALID_ARG;
    if (!(opts->angle_deg > 0.f && opts->angle_deg < 90.f) || opts->refine_iters < 0) return IMLOC_ERR_INVALID_ARG;
    TriParams p;
    memset(&p, 0, sizeof(p));
    p.u = u; p.v = v; p.conf = conf;
    p.stride = plane_stride;
    p.depth = depth_out;
    p.inliers = inliers_out;
    p.W = width; p.H = height; p.S = n_src;
    p.conf_min = opts->conf_min;
    const double tt = tan(static_cast<double>(opts->angle_deg) * M_PI / 180.0);
    p.tan2_thr = static_cast<float>(tt * tt);
    p.keep_more_than = opts->keep_more_than;
    p.refine_iters = opts->refine_iters;
    ray_matrix(*ref_cam, *ref_pose, p.M0, p.C0);
    for (int s = 0; s < n_src; ++s) {
        float C[3];
        ray_matrix(src_cams[s], src_poses[s], p.M[s], C);
        // C0 - C_s in FP64 before rounding
        for (int r = 0; r < 3; ++r) {
            double c0 = 0.0, cs = 0.0;
            for (int k = 0; k < 3; ++k) {
                c0 -= ref_pose->R[3 * k + r] * ref_pose->t[k];
                cs -= src_poses[s].R[3 * k + r] * src_poses[s].t[k];
            }
            p.W0[s][r] = static_cast<float>(c0 - cs);
        }
    }
    const int64_t n = static_cast<int64_t>(width) * height;
    const int64_t blocks = (n + 255) / 256;  // one CTA per 256 pixels
    if (blocks > INT32_MAX) return IMLOC_ERR_INVALID_ARG;
    const int grid = static_cast<int>(blocks);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_src <= 8) k_triangulate<8><<<grid, 256, 0, st>>>(p);
    else k_triangulate<16><<<grid, 256, 0, st>>>(p);
    IMLOC_CUDA_TRY(cudaGetLastError());
    return IMLOC_OK;
}

}  // extern "C"
