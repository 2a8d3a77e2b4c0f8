// p3p.cuh -- P3P for one minimal sample per thread (ImLoc Sec. 3.3 generates
// pose hypotheses with a P3P solver; this follows the Lambda Twist idea of
// Persson & Nordberg, ECCV 2018, written from the published mathematics).
//
// Unknowns: depths L = (l1, l2, l3) of the three points along unit bearings
// y_i.  The distance equations  L^T M_ij L = a_ij  (a_ij = |X_i - X_j|^2)
// give two homogeneous forms D1 = a23 M12 - a12 M23 and D2 = a23 M13 - a13 M23
// that vanish at every solution, as does D0 = D1 + g D2 for any g.  Choosing
// g as a real root of det(D1 + g D2) = 0 makes D0 a rank-2 indefinite form:
// it factors into two planes through the origin, sigma1 (e1.L)^2 + sigma2
// (e2.L)^2 = 0.  On each plane the depth with the largest normal component is
// eliminated, a second vanishing form gives a quadratic in the ratio of the
// other two, and the scale follows from the sum of the distance equations.
// The depths are polished by Newton on the distance equations (with
// double-float residuals when requested) and the pose is read off the triangle: R maps the world edge
// frame (X1-X2, X1-X3, cross) onto the camera one, t = l1 y1 - R X1.
#pragma once

#include "common.cuh"

namespace imloc {

struct Sym3 { float a00, a01, a02, a11, a12, a22; };

__device__ __forceinline__ float sym3_det(const Sym3& m) {
    return m.a00 * (m.a11 * m.a22 - m.a12 * m.a12) - m.a01 * (m.a01 * m.a22 - m.a12 * m.a02) +
           m.a02 * (m.a01 * m.a12 - m.a11 * m.a02);
}
// tr(adj(A) B) for symmetric A, B
__device__ __forceinline__ float sym3_adj_dot(const Sym3& A, const Sym3& B) {
    const float c00 = A.a11 * A.a22 - A.a12 * A.a12, c11 = A.a00 * A.a22 - A.a02 * A.a02, c22 = A.a00 * A.a11 - A.a01 * A.a01;
    const float c01 = A.a02 * A.a12 - A.a01 * A.a22, c02 = A.a01 * A.a12 - A.a02 * A.a11, c12 = A.a01 * A.a02 - A.a00 * A.a12;
    return c00 * B.a00 + c11 * B.a11 + c22 * B.a22 + 2.0f * (c01 * B.a01 + c02 * B.a02 + c12 * B.a12);
}
__device__ __forceinline__ Sym3 sym3_axpy(const Sym3& A, float g, const Sym3& B) {
    return Sym3{A.a00 + g * B.a00, A.a01 + g * B.a01, A.a02 + g * B.a02, A.a11 + g * B.a11, A.a12 + g * B.a12, A.a22 + g * B.a22};
}

// Real roots of c3 x^3 + c2 x^2 + c1 x + c0 (c3 != 0), Newton-polished.
__device__ int cubic_real_roots(float c3, float c2, float c1, float c0, float r[3]) {
    const float b = c2 / c3, c = c1 / c3, d = c0 / c3;
    const float p = c - b * b * (1.0f / 3.0f);
    const float q = (2.0f / 27.0f) * b * b * b - b * c * (1.0f / 3.0f) + d;
    const float disc = 0.25f * q * q + p * p * p * (1.0f / 27.0f);
    int n;
    if (disc > 0.0f) {
        const float sq = sqrtf(disc);
        const float u = cbrtf(-0.5f * q - copysignf(sq, q));
        r[0] = (u != 0.0f ? u - p / (3.0f * u) : 0.0f) - b * (1.0f / 3.0f);
        n = 1;
    } else {
        const float m = sqrtf(fmaxf(-p * (1.0f / 3.0f), 0.0f));
        float arg = (m > 0.0f) ? (-0.5f * q) / (m * m * m) : 0.0f;
        arg = fminf(1.0f, fmaxf(-1.0f, arg));
        const float th = acosf(arg) * (1.0f / 3.0f);
        r[0] = 2.0f * m * cosf(th) - b * (1.0f / 3.0f);
        r[1] = 2.0f * m * cosf(th - 2.0943951023931953f) - b * (1.0f / 3.0f);
        r[2] = 2.0f * m * cosf(th + 2.0943951023931953f) - b * (1.0f / 3.0f);
        n = 3;
    }
    for (int k = 0; k < n; ++k) {
        float x = r[k];
#pragma unroll
        for (int it = 0; it < 3; ++it) {
            const float f = ((x + b) * x + c) * x + d;
            const float df = (3.0f * x + 2.0f * b) * x + c;
            if (df != 0.0f) x -= f / df;
        }
        r[k] = x;
    }
    return n;
}

// Null vector of a symmetric rank-2 matrix: the longest cross product of two rows.
__device__ __forceinline__ void sym3_null(const Sym3& m, float v[3]) {
    const float r0[3] = {m.a00, m.a01, m.a02}, r1[3] = {m.a01, m.a11, m.a12}, r2[3] = {m.a02, m.a12, m.a22};
    float c[3][3];
    c[0][0] = r0[1] * r1[2] - r0[2] * r1[1]; c[0][1] = r0[2] * r1[0] - r0[0] * r1[2]; c[0][2] = r0[0] * r1[1] - r0[1] * r1[0];
    c[1][0] = r0[1] * r2[2] - r0[2] * r2[1]; c[1][1] = r0[2] * r2[0] - r0[0] * r2[2]; c[1][2] = r0[0] * r2[1] - r0[1] * r2[0];
    c[2][0] = r1[1] * r2[2] - r1[2] * r2[1]; c[2][1] = r1[2] * r2[0] - r1[0] * r2[2]; c[2][2] = r1[0] * r2[1] - r1[1] * r2[0];
    int best = 0;
    float bn = -1.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float nn = c[k][0] * c[k][0] + c[k][1] * c[k][1] + c[k][2] * c[k][2];
        if (nn > bn) { bn = nn; best = k; }
    }
    const float inv = rsqrtf(fmaxf(bn, 1e-37f));
    v[0] = c[best][0] * inv; v[1] = c[best][1] * inv; v[2] = c[best][2] * inv;
}

// Newton polish of the depths on the three distance equations: at most
// `iters` steps, stopping once every residual is below tol * a_ij.
template <typename T>
__device__ __forceinline__ void polish_depths(T L[3], const T a[3], const T b[3], int iters, T tol) {
    for (int it = 0; it < iters; ++it) {
        const T f0 = L[0] * L[0] + L[1] * L[1] - T(2) * b[0] * L[0] * L[1] - a[0];
        const T f1 = L[0] * L[0] + L[2] * L[2] - T(2) * b[1] * L[0] * L[2] - a[1];
        const T f2 = L[1] * L[1] + L[2] * L[2] - T(2) * b[2] * L[1] * L[2] - a[2];
        if (fabs(f0) <= tol * a[0] && fabs(f1) <= tol * a[1] && fabs(f2) <= tol * a[2]) return;
        const T j00 = T(2) * (L[0] - b[0] * L[1]), j01 = T(2) * (L[1] - b[0] * L[0]);
        const T j10 = T(2) * (L[0] - b[1] * L[2]), j12 = T(2) * (L[2] - b[1] * L[0]);
        const T j21 = T(2) * (L[1] - b[2] * L[2]), j22 = T(2) * (L[2] - b[2] * L[1]);
        // J = [[j00 j01 0], [j10 0 j12], [0 j21 j22]];  solve J d = f by Cramer
        const T det = j00 * (-j12 * j21) - j01 * (j10 * j22) ;
        if (det == T(0)) return;
        T inv;
        if constexpr (sizeof(T) == 4) {
            inv = T(1) / det;
        } else {
            // reciprocal: float32 seed, one Newton-Raphson step x (2 - det x) in FP64
            const T r0 = static_cast<T>(1.0f / static_cast<float>(det));
            inv = r0 * (T(2) - det * r0);
        }
        const T d0 = (f0 * (-j12 * j21) - j01 * (f1 * j22 - j12 * f2)) * inv;
        const T d1 = (j00 * (f1 * j22 - j12 * f2) - f0 * (j10 * j22)) * inv;
        const T d2 = (j00 * (-j21 * f1) - j01 * (j10 * f2) + f0 * (j10 * j21)) * inv;
        L[0] -= d0;
        L[1] -= d1;
        L[2] -= d2;
    }
}

// ---- double-float arithmetic --------------------------------------------
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// about 48 significant bits.  Error-free transformations: two_sum (Knuth),
// two_prod through the fused multiply-add (the rounding error of a*b is
// exactly fma(a, b, -a*b)).  Every operation is written with the _rn
// intrinsics so that the compiler neither contracts nor reassociates them.
// The Newton polish of the P3P depths needs the residuals of the distance
// equations to far more than FP32 precision (they cancel terms of size
// depth^2 down to the triangle's squared sides); double-float gives that on
// the FP32 pipe, which this GPU runs at 64 times its FP64 rate.
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfloat{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return dfloat{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat{-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const dfloat p = df_two_prod(a.hi, b.hi);
    return df_fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

// Unit bearing of pixel (px, py): ((px - cx) / fx, (py - cy) / fy, 1) / norm,
// in double-float (1/fx, 1/fy given as double-floats).
__device__ __forceinline__ void bearing_df(float px, float py, float cx, float cy, dfloat ifx, dfloat ify,
                                           dfloat out[3]) {
    const dfloat ex = df_mul(df_two_sum(px, -cx), ifx);
    const dfloat ey = df_mul(df_two_sum(py, -cy), ify);
    const dfloat n2 = df_add(df_add(df_mul(ex, ex), df_mul(ey, ey)), dfloat{1.0f, 0.0f});
    // 1 / sqrt(n2): float seed r0, rho = 1 - n2 r0^2 (small, in double-float),
    // r = r0 (1 + rho / 2 + 3 rho^2 / 8) (binomial series; the next term is
    // below 1e-18 for the seed's accuracy)
    const float r0 = rsqrtf(n2.hi);
    const dfloat t = df_mul(n2, df_two_prod(r0, r0));
    const float rho = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    const float corr = __fmul_rn(r0, __fmul_rn(rho, __fmaf_rn(0.375f, rho, 0.5f)));
    const dfloat r = df_fast_two_sum(r0, corr);
    out[0] = df_mul(ex, r);
    out[1] = df_mul(ey, r);
    out[2] = r;
}

// Li^2 + Lj^2 - 2 b Li Lj - a for float depths and double-float b, a: the
// terms of size Li^2 cancel exactly (error-free products and sums), so the
// result is accurate to ~1e-14 of them.
__device__ __forceinline__ float dist_residual_df(float Li, float Lj, dfloat b, dfloat a) {
    const dfloat bq = df_mul(b, df_two_prod(Li, Lj));
    dfloat s = df_add(df_two_prod(Li, Li), df_two_prod(Lj, Lj));
    s = df_add(s, dfloat{-2.0f * bq.hi, -2.0f * bq.lo});
    s = df_add(s, df_neg(a));
    return __fadd_rn(s.hi, s.lo);
}

// Newton polish of float depths with double-float residuals (Jacobian and
// step in FP32): at most `iters` steps, stopping once a step no longer
// changes the depths beyond float resolution.
__device__ __forceinline__ void polish_depths_df(float L[3], const dfloat a[3], const dfloat b[3], int iters) {
    for (int it = 0; it < iters; ++it) {
        const float f0 = dist_residual_df(L[0], L[1], b[0], a[0]);
        const float f1 = dist_residual_df(L[0], L[2], b[1], a[1]);
        const float f2 = dist_residual_df(L[1], L[2], b[2], a[2]);
        const float j00 = 2.0f * (L[0] - b[0].hi * L[1]), j01 = 2.0f * (L[1] - b[0].hi * L[0]);
        const float j10 = 2.0f * (L[0] - b[1].hi * L[2]), j12 = 2.0f * (L[2] - b[1].hi * L[0]);
        const float j21 = 2.0f * (L[1] - b[2].hi * L[2]), j22 = 2.0f * (L[2] - b[2].hi * L[1]);
        // J = [[j00 j01 0], [j10 0 j12], [0 j21 j22]];  solve J d = f by Cramer
        const float det = j00 * (-j12 * j21) - j01 * (j10 * j22);
        if (det == 0.0f) return;
        const float inv = 1.0f / det;
        const float d0 = (f0 * (-j12 * j21) - j01 * (f1 * j22 - j12 * f2)) * inv;
        const float d1 = (j00 * (f1 * j22 - j12 * f2) - f0 * (j10 * j22)) * inv;
        const float d2 = (j00 * (-j21 * f1) - j01 * (j10 * f2) + f0 * (j10 * j21)) * inv;
        L[0] -= d0;
        L[1] -= d1;
        L[2] -= d2;
        const float tiny = 6e-8f;  // 2^-24: the step is below the depths' float resolution
        if (fabsf(d0) <= tiny * fabsf(L[0]) && fabsf(d1) <= tiny * fabsf(L[1]) && fabsf(d2) <= tiny * fabsf(L[2]))
            return;
    }
}

// Pose from depths: R (X1-X2, X1-X3, cross) = (C1-C2, C1-C3, cross), t = C1 - R X1.
template <typename T, typename B>
__device__ __forceinline__ bool pose_from_depths(const T L[3], const B y[3][3], const float X[3][3], float Rout[9],
                                                 float tout[3]) {
    T C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) C[i][a] = L[i] * T(y[i][a]);
    T v1[3], v2[3], c1[3], c2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v1[a] = T(X[0][a]) - T(X[1][a]);
        v2[a] = T(X[0][a]) - T(X[2][a]);
        c1[a] = C[0][a] - C[1][a];
        c2[a] = C[0][a] - C[2][a];
    }
    const T v3[3] = {v1[1] * v2[2] - v1[2] * v2[1], v1[2] * v2[0] - v1[0] * v2[2], v1[0] * v2[1] - v1[1] * v2[0]};
    const T c3[3] = {c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2], c1[0] * c2[1] - c1[1] * c2[0]};
    // V = [v1 v2 v3] (columns); V^-1 = adj(V) / det(V); rows of V^-1 are (v2 x v3, v3 x v1, v1 x v2) / det
    const T det = v1[0] * (v2[1] * v3[2] - v2[2] * v3[1]) - v2[0] * (v1[1] * v3[2] - v1[2] * v3[1]) +
                  v3[0] * (v1[1] * v2[2] - v1[2] * v2[1]);
    if (!(det != T(0))) return false;
    const T id = T(1) / det;
    T w[3][3];  // rows of V^-1
    w[0][0] = (v2[1] * v3[2] - v2[2] * v3[1]) * id; w[0][1] = (v2[2] * v3[0] - v2[0] * v3[2]) * id; w[0][2] = (v2[0] * v3[1] - v2[1] * v3[0]) * id;
    w[1][0] = (v3[1] * v1[2] - v3[2] * v1[1]) * id; w[1][1] = (v3[2] * v1[0] - v3[0] * v1[2]) * id; w[1][2] = (v3[0] * v1[1] - v3[1] * v1[0]) * id;
    w[2][0] = (v1[1] * v2[2] - v1[2] * v2[1]) * id; w[2][1] = (v1[2] * v2[0] - v1[0] * v2[2]) * id; w[2][2] = (v1[0] * v2[1] - v1[1] * v2[0]) * id;
    T R[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) R[3 * r + c] = c1[r] * w[0][c] + c2[r] * w[1][c] + c3[r] * w[2][c];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rout[k] = static_cast<float>(R[k]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
        tout[r] = static_cast<float>(C[0][r] - (R[3 * r] * T(X[0][0]) + R[3 * r + 1] * T(X[0][1]) + R[3 * r + 2] * T(X[0][2])));
    return true;
}

// One Newton-Schulz step towards the nearest rotation: R <- R (3 I - R^T R) / 2
// (the triangle-frame pose is a rotation up to float32 rounding).
template <typename T>
__device__ __forceinline__ void orthonormalize(T R[9]) {
    T G[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) G[3 * i + j] = R[i] * R[j] + R[3 + i] * R[3 + j] + R[6 + i] * R[6 + j];
    T N[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T m0 = (0 == j ? T(3) : T(0)) - G[j], m1 = (1 == j ? T(3) : T(0)) - G[3 + j],
                    m2 = (2 == j ? T(3) : T(0)) - G[6 + j];
            N[3 * i + j] = T(0.5) * (R[3 * i] * m0 + R[3 * i + 1] * m1 + R[3 * i + 2] * m2);
        }
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = N[k];
}

// Solve one P3P instance.  y: unit bearings (float32), yd: the same bearings
// in double-float (used, with double-float squared distances, by the Newton
// polish when non-null), X: world points.  Returns the number of poses
// (<= 4), sorted by ascending depth of the first point.
__device__ int p3p_solve(const float y[3][3], const dfloat (*yd)[3], const float X[3][3], PoseF out[4],
                         float l1_out[4]) {
    const bool fp64_polish = yd != nullptr;
    float a12 = 0.f, a13 = 0.f, a23 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float d12 = X[0][k] - X[1][k], d13 = X[0][k] - X[2][k], d23 = X[1][k] - X[2][k];
        a12 = fmaf(d12, d12, a12);
        a13 = fmaf(d13, d13, a13);
        a23 = fmaf(d23, d23, a23);
    }
    if (!(a12 > 0.f) || !(a13 > 0.f) || !(a23 > 0.f)) return 0;
    const float b12 = y[0][0] * y[1][0] + y[0][1] * y[1][1] + y[0][2] * y[1][2];
    const float b13 = y[0][0] * y[2][0] + y[0][1] * y[2][1] + y[0][2] * y[2][2];
    const float b23 = y[1][0] * y[2][0] + y[1][1] * y[2][1] + y[1][2] * y[2][2];
    // scale the squared distances to <= 1 (depths scale by sqrt)
    const float amax = fmaxf(a12, fmaxf(a13, a23));
    const float sa = 1.0f / amax;
    const float A12 = a12 * sa, A13 = a13 * sa, A23 = a23 * sa;
    const Sym3 D1{A23, -A23 * b12, 0.f, A23 - A12, A12 * b23, -A12};
    const Sym3 D2{A23, 0.f, -A23 * b13, -A13, A13 * b23, A23 - A13};
    const float c3 = sym3_det(D2), c2 = sym3_adj_dot(D2, D1), c1 = sym3_adj_dot(D1, D2), c0 = sym3_det(D1);
    float roots[3];
    int nr = 0;
    const float cm = fmaxf(fmaxf(fabsf(c0), fabsf(c1)), fmaxf(fabsf(c2), fabsf(c3)));
    if (fabsf(c3) > 1e-7f * cm) nr = cubic_real_roots(c3, c2, c1, c0, roots);
    // pick the root that makes D0 most clearly indefinite (sigma1 sigma2 < 0)
    float best_q = 0.f, g = 0.f;
    Sym3 D0{};
    bool have = false;
    for (int k = 0; k < nr; ++k) {
        const Sym3 M = sym3_axpy(D1, roots[k], D2);
        const float minors = M.a00 * M.a11 - M.a01 * M.a01 + M.a00 * M.a22 - M.a02 * M.a02 + M.a11 * M.a22 - M.a12 * M.a12;
        const float nrm = M.a00 * M.a00 + M.a11 * M.a11 + M.a22 * M.a22 + 2.f * (M.a01 * M.a01 + M.a02 * M.a02 + M.a12 * M.a12);
        const float qual = -minors / fmaxf(nrm, 1e-30f);
        if (qual > best_q) { best_q = qual; g = roots[k]; D0 = M; have = true; }
    }
    if (!have) {
        // det(D2) ~ 0: D2 itself is the degenerate form (g -> infinity)
        const float minors = D2.a00 * D2.a11 - D2.a01 * D2.a01 + D2.a00 * D2.a22 - D2.a02 * D2.a02 + D2.a11 * D2.a22 - D2.a12 * D2.a12;
        if (!(minors < 0.f)) return 0;
        D0 = D2;
        g = 1e30f;
    }
    // eigen-decomposition of the rank-2 D0: sigma1 > 0 > sigma2
    const float tr = D0.a00 + D0.a11 + D0.a22;
    const float minors = D0.a00 * D0.a11 - D0.a01 * D0.a01 + D0.a00 * D0.a22 - D0.a02 * D0.a02 + D0.a11 * D0.a22 - D0.a12 * D0.a12;
    const float disc = sqrtf(fmaxf(tr * tr - 4.f * minors, 0.f));
    const float s1 = 0.5f * (tr + disc), s2 = 0.5f * (tr - disc);
    if (!(s1 > 0.f) || !(s2 < 0.f)) return 0;
    float e3[3], e1[3];
    sym3_null(D0, e3);
    const Sym3 Ms{D0.a00 - s1, D0.a01, D0.a02, D0.a11 - s1, D0.a12, D0.a22 - s1};
    sym3_null(Ms, e1);
    const float e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
    const float s = sqrtf(-s2 / s1);
    const Sym3& D = (fabsf(g) <= 1.0f) ? D2 : D1;

    float Ls[4][3];
    int ns = 0;
    const float asum = A12 + A13 + A23;
#pragma unroll
    for (int sign = 0; sign < 2; ++sign) {
        const float ss = sign ? -s : s;
        const float n[3] = {e1[0] - ss * e2[0], e1[1] - ss * e2[1], e1[2] - ss * e2[2]};
        // on the plane n.L = 0 eliminate the depth with the largest |n_k|;
        // the other two, (l_i, l_j) = l_j (tau, 1), stay free
        int k = 0;
        if (fabsf(n[1]) > fabsf(n[k])) k = 1;
        if (fabsf(n[2]) > fabsf(n[k])) k = 2;
        const int i = (k == 0) ? 1 : 0, j = (k == 2) ? 1 : 2;
        if (!(fabsf(n[k]) > 0.f)) continue;
        const float ci = -n[i] / n[k], cj = -n[j] / n[k];  // l_k = ci l_i + cj l_j
        // A = columns (d l / d l_i, d l / d l_j); Q = A^T D A restricted to the plane
        float ai[3] = {0.f, 0.f, 0.f}, aj[3] = {0.f, 0.f, 0.f};
        ai[i] = 1.f; ai[k] = ci;
        aj[j] = 1.f; aj[k] = cj;
        const float Dai[3] = {D.a00 * ai[0] + D.a01 * ai[1] + D.a02 * ai[2], D.a01 * ai[0] + D.a11 * ai[1] + D.a12 * ai[2],
                              D.a02 * ai[0] + D.a12 * ai[1] + D.a22 * ai[2]};
        const float Daj[3] = {D.a00 * aj[0] + D.a01 * aj[1] + D.a02 * aj[2], D.a01 * aj[0] + D.a11 * aj[1] + D.a12 * aj[2],
                              D.a02 * aj[0] + D.a12 * aj[1] + D.a22 * aj[2]};
        const float q00 = ai[0] * Dai[0] + ai[1] * Dai[1] + ai[2] * Dai[2];
        const float q01 = ai[0] * Daj[0] + ai[1] * Daj[1] + ai[2] * Daj[2];
        const float q11 = aj[0] * Daj[0] + aj[1] * Daj[1] + aj[2] * Daj[2];
        const float dq = q01 * q01 - q00 * q11;
        if (dq < 0.f || q00 == 0.f) continue;
        const float sq = sqrtf(dq);
        // stable roots of q00 tau^2 + 2 q01 tau + q11 = 0, tau = l_i / l_j
        const float tmp = -q01 - copysignf(sq, q01);
        const float taus[2] = {tmp / q00, (tmp != 0.f) ? q11 / tmp : 0.f};
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float tau = taus[r];
            if (!(tau > 0.f)) continue;
            const float v[3] = {tau * ai[0] + aj[0], tau * ai[1] + aj[1], tau * ai[2] + aj[2]};
            // scale from the sum of the three distance equations (all solutions satisfy it)
            const float den = (v[0] * v[0] + v[1] * v[1] - 2.f * b12 * v[0] * v[1]) +
                              (v[0] * v[0] + v[2] * v[2] - 2.f * b13 * v[0] * v[2]) +
                              (v[1] * v[1] + v[2] * v[2] - 2.f * b23 * v[1] * v[2]);
            if (!(den > 0.f)) continue;
            const float lj = sqrtf(asum / den);
            const float l1 = v[0] * lj, l2 = v[1] * lj, l3 = v[2] * lj;
            if (!(l1 > 0.f) || !(l2 > 0.f) || !(l3 > 0.f)) continue;
            if (ns < 4) {
                Ls[ns][0] = l1; Ls[ns][1] = l2; Ls[ns][2] = l3;
                ++ns;
            }
        }
    }
    // rescale, polish, validate, pose
    const float scale = sqrtf(amax);
    // the distance equations in double-float for the extended-precision polish
    dfloat a_df[3], b_df[3];
    if (fp64_polish) {
        const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            dfloat acc{0.0f, 0.0f};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const dfloat dc = df_two_sum(X[pi[e]][c], -X[pj[e]][c]);
                acc = df_add(acc, df_mul(dc, dc));
            }
            a_df[e] = acc;
            b_df[e] = df_add(df_add(df_mul(yd[pi[e]][0], yd[pj[e]][0]), df_mul(yd[pi[e]][1], yd[pj[e]][1])),
                             df_mul(yd[pi[e]][2], yd[pj[e]][2]));
        }
    }
    int nout = 0;
    for (int k = 0; k < ns; ++k) {
        bool good;
        float Lf[3];
        if (fp64_polish) {
            float L[3] = {Ls[k][0] * scale, Ls[k][1] * scale, Ls[k][2] * scale};
            polish_depths_df(L, a_df, b_df, 4);
            const float f0 = dist_residual_df(L[0], L[1], b_df[0], a_df[0]);
            const float f1 = dist_residual_df(L[0], L[2], b_df[1], a_df[1]);
            const float f2 = dist_residual_df(L[1], L[2], b_df[2], a_df[2]);
            good = L[0] > 0 && L[1] > 0 && L[2] > 0 && fabsf(f0) <= 1e-4f * a_df[0].hi &&
                   fabsf(f1) <= 1e-4f * a_df[1].hi && fabsf(f2) <= 1e-4f * a_df[2].hi;
            if (good) {
                // the pose from the polished depths in float32 (the poses are scored in float32)
                good = pose_from_depths<float, float>(L, y, X, out[nout].R, out[nout].t);
                if (good) orthonormalize(out[nout].R);
            }
            Lf[0] = L[0];
        } else {
            float L[3] = {Ls[k][0] * scale, Ls[k][1] * scale, Ls[k][2] * scale};
            const float a[3] = {a12, a13, a23}, b[3] = {b12, b13, b23};
            polish_depths<float>(L, a, b, 2, 1e-6f);
            const float f0 = L[0] * L[0] + L[1] * L[1] - 2.0f * b[0] * L[0] * L[1] - a[0];
            const float f1 = L[0] * L[0] + L[2] * L[2] - 2.0f * b[1] * L[0] * L[2] - a[1];
            const float f2 = L[1] * L[1] + L[2] * L[2] - 2.0f * b[2] * L[1] * L[2] - a[2];
            good = L[0] > 0 && L[1] > 0 && L[2] > 0 && fabsf(f0) <= 1e-3f * a[0] && fabsf(f1) <= 1e-3f * a[1] &&
                   fabsf(f2) <= 1e-3f * a[2];
            if (good) good = pose_from_depths<float, float>(L, y, X, out[nout].R, out[nout].t);
            if (good) orthonormalize(out[nout].R);
            Lf[0] = L[0];
        }
        if (!good) continue;
        bool dup = false;
        for (int j = 0; j < nout; ++j)
            if (fabsf(l1_out[j] - Lf[0]) <= 1e-5f * Lf[0]) dup = true;
        if (dup) continue;
        l1_out[nout] = Lf[0];
        ++nout;
    }
    // ascending depth of the first point
    for (int i = 1; i < nout; ++i)
        for (int j = i; j > 0 && l1_out[j] < l1_out[j - 1]; --j) {
            const float tl = l1_out[j]; l1_out[j] = l1_out[j - 1]; l1_out[j - 1] = tl;
            const PoseF tp = out[j]; out[j] = out[j - 1]; out[j - 1] = tp;
        }
    return nout;
}

}  // namespace imloc
