// gp3p.cuh -- generalized P3P on the GPU (one minimal sample per thread, FP64):
// the rig pose that puts three world points on three rays of a multi-camera
// rig (ImLoc supplementary "LaMAR HoloLens Results": a GPU generalized
// absolute pose estimator for queries taken by a camera rig).
//
// A rigid motion keeps distances, so the depths lambda_i along the rays
// o_i + lambda_i d_i (rig frame, |d_i| = 1) satisfy, for each pair i < j,
//   lambda_i^2 + lambda_j^2 - 2 c_ij lambda_i lambda_j + 2 a_ij lambda_i
//     - 2 b_ij lambda_j + e_ij = 0,
//   c_ij = d_i.d_j, a_ij = d_i.(o_i - o_j), b_ij = d_j.(o_i - o_j),
//   e_ij = |o_i - o_j|^2 - |X_i - X_j|^2.
// Pairs (1,2) and (1,3) are monic quadratics in lambda_2 and lambda_3 whose
// coefficients are polynomials in lambda_1; pair (2,3) minus both leaves a
// bilinear relation giving lambda_3 from lambda_2; substituting it into pair
// (1,3) gives a second quadratic in lambda_2, and the resultant of the two
// quadratics is a polynomial of degree 8 in lambda_1 (at most 8 poses).
//
// Root finding is bracketing, not a full polynomial solve: every real
// solution has real lambda_2 and lambda_3, so lambda_1 lies where the
// discriminants of both quadratics are >= 0 -- a bounded interval (the rays
// are not parallel).  The octic, rewritten in mu over that interval, is
// scanned at Chebyshev nodes (roots crowd towards the interval's ends); each
// sign change brackets a root, and a cell whose ends agree in sign but not in
// slope is split at the extremum (two close roots).  Each root is refined to
// float precision, lambda_2 and lambda_3 follow by back-substitution, and
// Newton on the three distance equations (FP64) polishes the triple.  The
// scan and the root refinement run in double-float on the FP32 pipe (this
// GPU's FP64 rate is 1/64 of FP32); the coefficients, the back-substitution
// and the polish are FP64.  The pose comes from the two triangles'
// orthonormal frames.  Roots that touch zero without a sign change (a double
// solution: an ill-conditioned, degenerate configuration) are not reported.
#pragma once

#include <stdint.h>

namespace imloc {

constexpr int kGp3pGrid = 64;      // sign-change grid over the feasible interval
constexpr int kGp3pMaxSol = 8;

struct Gp3pSol {
    int n;
    double lam[kGp3pMaxSol][3];
};

// p(x) = sum_k c[k] x^k
template <int D>
__device__ __forceinline__ double gp_eval(const double (&c)[D + 1], double x) {
    double a = c[D];
#pragma unroll
    for (int k = D - 1; k >= 0; --k) a = fma(a, x, c[k]);
    return a;
}
// out = a * b (degrees A, B)
template <int A, int B>
__device__ __forceinline__ void gp_mul(const double (&a)[A + 1], const double (&b)[B + 1], double (&out)[A + B + 1]) {
#pragma unroll
    for (int k = 0; k <= A + B; ++k) out[k] = 0.0;
#pragma unroll
    for (int i = 0; i <= A; ++i)
#pragma unroll
        for (int j = 0; j <= B; ++j) out[i + j] = fma(a[i], b[j], out[i + j]);
}
__device__ __forceinline__ double dot3d(const double* a, const double* b) {
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// interval where alpha x^2 + 2 beta x + gamma >= 0 for alpha < 0; false if empty
__device__ __forceinline__ bool gp_feasible(double alpha, double beta, double gamma, double& lo, double& hi) {
    if (!(alpha < 0.0)) return false;  // parallel rays: no bounded interval
    const double disc = beta * beta - alpha * gamma;
    if (disc < 0.0) return false;
    const double s = sqrt(disc);
    const double x1 = (-beta + s) / alpha, x2 = (-beta - s) / alpha;
    lo = fmin(x1, x2);
    hi = fmax(x1, x2);
    return true;
}

// the three distance residuals and their Jacobian (each row has two nonzeros)
__device__ __forceinline__ void gp_system(const double o[3][3], const double d[3][3], const double D2[3],
                                          const double L[3], double f[3], double J[3][3]) {
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int i = pi[e], j = pj[e];
        double v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = (o[i][a] - o[j][a]) + L[i] * d[i][a] - L[j] * d[j][a];
        f[e] = dot3d(v, v) - D2[e];
        J[e][0] = J[e][1] = J[e][2] = 0.0;
        J[e][i] = 2.0 * dot3d(v, d[i]);
        J[e][j] = -2.0 * dot3d(v, d[j]);
    }
}

__device__ __forceinline__ bool gp_solve3(const double A[3][3], const double b[3], double x[3]) {
    const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    const double id = 1.0 / det;
    const double inv[3][3] = {
        {c00 * id, (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id, (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id},
        {c01 * id, (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id, (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id},
        {c02 * id, (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id, (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id}};
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = inv[r][0] * b[0] + inv[r][1] * b[1] + inv[r][2] * b[2];
    return true;
}

// Everything the root search and the back-substitution need for one minimal
// set (coefficient polynomials in lambda_1, ascending).
struct Gp3pSys {
    double oct[9];
    double f2[3], f1[4], f0[5];   // F(l2) = f2 l2^2 + f1 l2 + f0
    double q[3], g1[2];           // G(l2) = l2^2 + g1 l2 + q
    double B[2], C[2], E[3];      // l3 = -(B l2 + E) / (A l2 + C)
    double r[2], s[3];            // l3^2 - 2 r l3 + s (pair 1,3)
    double A;
    double D2[3];
    double lo, hi;                // feasible lambda_1 (padded)
};

// A bracket [l, u] of one root of the octic (p(l) = pl has the other sign).
struct Gp3pBracket {
    double l, u, pl;
};

// Coefficients and the feasible interval; false if no real solution can exist.
__device__ inline bool gp3p_setup(const double o[3][3], const double d[3][3], const double X[3][3], Gp3pSys& S) {
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
    double c[3], a[3], b[3], e[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = pi[k], j = pj[k];
        double oij[3], x[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            oij[m] = o[i][m] - o[j][m];
            x[m] = X[i][m] - X[j][m];
        }
        S.D2[k] = dot3d(x, x);
        c[k] = dot3d(d[i], d[j]);
        a[k] = dot3d(d[i], oij);
        b[k] = dot3d(d[j], oij);
        e[k] = dot3d(oij, oij) - S.D2[k];
    }
    // feasible lambda_1: real lambda_2 (pair 1,2) and real lambda_3 (pair 1,3)
    double lo2, hi2, lo3, hi3;
    if (!gp_feasible(c[0] * c[0] - 1.0, c[0] * b[0] - a[0], b[0] * b[0] - e[0], lo2, hi2)) return false;
    if (!gp_feasible(c[1] * c[1] - 1.0, c[1] * b[1] - a[1], b[1] * b[1] - e[1], lo3, hi3)) return false;
    double lo = fmax(fmax(lo2, lo3), 0.0), hi = fmin(hi2, hi3);
    if (!(hi > lo)) return false;
    const double pad = 1e-9 * (hi - lo) + 1e-12 * hi;
    S.lo = fmax(lo - pad, 0.0);
    S.hi = hi + pad;

    const double p[2] = {b[0], c[0]};  // G: l2^2 - 2 p l2 + q
    S.q[0] = e[0];
    S.q[1] = 2.0 * a[0];
    S.q[2] = 1.0;
    S.r[0] = b[1];
    S.r[1] = c[1];
    S.s[0] = e[1];
    S.s[1] = 2.0 * a[1];
    S.s[2] = 1.0;
    S.A = -2.0 * c[2];
    S.B[0] = 2.0 * (p[0] + a[2]);
    S.B[1] = 2.0 * p[1];
    S.C[0] = 2.0 * (S.r[0] - b[2]);
    S.C[1] = 2.0 * S.r[1];
    S.E[0] = e[2] - S.q[0] - S.s[0];
    S.E[1] = -S.q[1] - S.s[1];
    S.E[2] = -S.q[2] - S.s[2];
    const double A = S.A;
    {
        double BB[3], rB[3];
        gp_mul<1, 1>(S.B, S.B, BB);
        gp_mul<1, 1>(S.r, S.B, rB);
#pragma unroll
        for (int k = 0; k < 3; ++k) S.f2[k] = BB[k] + 2.0 * A * rB[k] + A * A * S.s[k];
        double BE[4], BC[3], rBC[4], rE[4], sC[4];
        gp_mul<1, 2>(S.B, S.E, BE);
        gp_mul<1, 1>(S.B, S.C, BC);
        gp_mul<1, 2>(S.r, BC, rBC);
        gp_mul<1, 2>(S.r, S.E, rE);
        gp_mul<2, 1>(S.s, S.C, sC);
#pragma unroll
        for (int k = 0; k < 4; ++k) S.f1[k] = 2.0 * (BE[k] + rBC[k] + A * rE[k] + A * sC[k]);
        double EE[5], rEC[5], CC[3], sCC[5];
        gp_mul<2, 2>(S.E, S.E, EE);
        gp_mul<3, 1>(rE, S.C, rEC);
        gp_mul<1, 1>(S.C, S.C, CC);
        gp_mul<2, 2>(S.s, CC, sCC);
#pragma unroll
        for (int k = 0; k < 5; ++k) S.f0[k] = EE[k] + 2.0 * rEC[k] + sCC[k];
    }
    S.g1[0] = -2.0 * p[0];
    S.g1[1] = -2.0 * p[1];
    {
        // resultant (f2 g0 - f0)^2 - (f2 g1 - f1)(f1 g0 - f0 g1)
        double t1[5], t2[4], t3[6], tmp5[5], tmp4[4], tmp6[6], f0g1[6];
        gp_mul<2, 2>(S.f2, S.q, tmp5);
#pragma unroll
        for (int k = 0; k < 5; ++k) t1[k] = tmp5[k] - S.f0[k];
        gp_mul<2, 1>(S.f2, S.g1, tmp4);
#pragma unroll
        for (int k = 0; k < 4; ++k) t2[k] = tmp4[k] - S.f1[k];
        gp_mul<3, 2>(S.f1, S.q, tmp6);
        gp_mul<4, 1>(S.f0, S.g1, f0g1);
#pragma unroll
        for (int k = 0; k < 6; ++k) t3[k] = tmp6[k] - f0g1[k];
        double t11[9], t23[9];
        gp_mul<4, 4>(t1, t1, t11);
        gp_mul<3, 5>(t2, t3, t23);
#pragma unroll
        for (int k = 0; k < 9; ++k) S.oct[k] = t11[k] - t23[k];
    }
    return true;
}

// Double-float (float hi + lo, ~48-bit significand on the FP32 pipe; this
// GPU's FP64 rate is 1/64 of FP32) for the grid scan of the octic.
struct gdf {
    float hi, lo;
};
__device__ __forceinline__ gdf gdf_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return gdf{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ gdf gdf_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return gdf{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ gdf gdf_add(gdf a, gdf b) {
    const gdf s = gdf_two_sum(a.hi, b.hi);
    return gdf_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ gdf gdf_mul_f(gdf a, float b) {  // a * b, b exact in float
    const float p = __fmul_rn(a.hi, b);
    return gdf_fast_two_sum(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
__device__ __forceinline__ bool gdf_neg(gdf a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f); }
__device__ __forceinline__ bool gdf_zero(gdf a) { return a.hi == 0.0f && a.lo == 0.0f; }

// p, p' and p''/2 at mu of the polynomial with double-float coefficients c[0..8]
__device__ __forceinline__ void gdf_horner(const gdf (&c)[9], float mu, gdf& p, gdf& dp, gdf& ddp, bool second) {
    p = c[8];
    dp = gdf{0.0f, 0.0f};
    ddp = gdf{0.0f, 0.0f};
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        if (second) ddp = gdf_add(gdf_mul_f(ddp, mu), dp);
        dp = gdf_add(gdf_mul_f(dp, mu), p);
        p = gdf_add(gdf_mul_f(p, mu), c[k]);
    }
}

// Root brackets of the octic over the feasible interval, ascending: sign
// changes between grid nodes, and cells whose ends agree in sign but not in
// slope split at the extremum of p (two close roots).  The octic is first
// rewritten in mu, x = mid + half mu (Taylor shift in FP64, coefficients
// scaled to a largest magnitude of 1) and scanned in double-float at the
// Chebyshev nodes mu_j = -cos(pi j / G) (roots crowd towards the ends of the
// interval, where lambda_2 or lambda_3 turns complex).  Brackets are
// returned in x.  Returns the count.
// The octic in mu, x = mid + half mu: Taylor shift in FP64, coefficients
// scaled to a largest magnitude of 1, as double-floats; false if degenerate.
__device__ inline bool gp3p_shifted(const Gp3pSys& S, double mid, double half, gdf (&c)[9]) {
    {
        double b[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) b[k] = S.oct[k];
        // coefficients of p(mid + y): repeated synthetic division by (y - mid)
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int k = 7; k >= i; --k) b[k] = fma(mid, b[k + 1], b[k]);
        double h = 1.0, mx = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            b[k] *= h;
            h *= half;
            mx = fmax(mx, fabs(b[k]));
        }
        if (!(mx > 0.0) || !isfinite(mx)) return false;
        const double inv = 1.0 / mx;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double v = b[k] * inv;
            const float hi = static_cast<float>(v);
            c[k] = gdf{hi, static_cast<float>(v - static_cast<double>(hi))};
        }
    }
    return true;
}

__device__ inline int gp3p_brackets(const Gp3pSys& S, Gp3pBracket* br, int nmax) {
    const double mid = 0.5 * (S.lo + S.hi), half = 0.5 * (S.hi - S.lo);
    gdf c[9];
    if (!gp3p_shifted(S, mid, half, c)) return 0;
    auto x_of = [&](float mu) { return mu == -1.0f ? S.lo : (mu == 1.0f ? S.hi : mid + half * static_cast<double>(mu)); };
    int n = 0;
    float ma = -1.0f;
    gdf pa, dpa, dd;
    gdf_horner(c, ma, pa, dpa, dd, false);
    for (int gi = 1; gi <= kGp3pGrid && n < nmax; ++gi) {
        const float mb = gi == kGp3pGrid ? 1.0f : -cospif(static_cast<float>(gi) * (1.0f / kGp3pGrid));
        gdf pb, dpb;
        gdf_horner(c, mb, pb, dpb, dd, false);
        if (gdf_zero(pa)) {
            br[n++] = Gp3pBracket{x_of(ma), x_of(ma), 0.0};
        } else if (!gdf_zero(pb) && gdf_neg(pa) != gdf_neg(pb)) {
            br[n++] = Gp3pBracket{x_of(ma), x_of(mb), gdf_neg(pa) ? -1.0 : 1.0};
        } else if (!gdf_zero(pb) && gdf_neg(dpa) != gdf_neg(dpb)) {
            // the extremum: Newton on p' kept inside the bracket where p' changes sign
            float l = ma, u = mb, m = 0.5f * (ma + mb);
            for (int it = 0; it < 20; ++it) {
                gdf p0, p1, p2;
                gdf_horner(c, m, p0, p1, p2, true);
                if (gdf_neg(p1) == gdf_neg(dpa)) l = m; else u = m;
                const float d2 = 2.0f * __fadd_rn(p2.hi, p2.lo);  // the recurrence gives p'' / 2
                float mn = m - __fadd_rn(p1.hi, p1.lo) / d2;
                if (!(mn > l && mn < u)) mn = 0.5f * (l + u);
                const bool conv = mn == m || u - l <= 4e-7f * fabsf(u) + 1e-30f;
                m = mn;
                if (conv) break;
            }
            gdf pe, de;
            gdf_horner(c, m, pe, de, dd, false);
            if (gdf_neg(pe) != gdf_neg(pa) && !gdf_zero(pe) && n + 2 <= nmax && m > ma && m < mb) {
                br[n++] = Gp3pBracket{x_of(ma), x_of(m), gdf_neg(pa) ? -1.0 : 1.0};
                br[n++] = Gp3pBracket{x_of(m), x_of(mb), gdf_neg(pe) ? -1.0 : 1.0};
            }
        }
        ma = mb;
        pa = pb;
        dpa = dpb;
    }
    return n;
}

// The root in a bracket, lambda_2 and lambda_3 by back-substitution (the
// common root of F and G, then the bilinear relation), Newton on the three
// distance equations; true if the triple is a solution with positive depths.
__device__ inline bool gp3p_finish(const Gp3pSys& S, const double o[3][3], const double d[3][3],
                                   const Gp3pBracket& b, double L[3]) {
    // the root to float precision in mu (double-float octic, Newton kept in the
    // bracket); the Newton steps on the distance equations below finish it
    double l1 = b.l;
    if (b.u > b.l) {
        const double mid = 0.5 * (S.lo + S.hi), half = 0.5 * (S.hi - S.lo);
        gdf c[9];
        if (!gp3p_shifted(S, mid, half, c)) return false;
        float l = static_cast<float>((b.l - mid) / half), u = static_cast<float>((b.u - mid) / half);
        const bool neg_l = b.pl < 0.0;
        float m = 0.5f * (l + u);
        for (int it = 0; it < 40; ++it) {
            gdf p, dp, dd;
            gdf_horner(c, m, p, dp, dd, false);
            if (gdf_zero(p)) break;
            if (gdf_neg(p) == neg_l) l = m; else u = m;
            float mn = m - __fadd_rn(p.hi, p.lo) / __fadd_rn(dp.hi, dp.lo);
            if (!(mn > l && mn < u)) mn = 0.5f * (l + u);
            const bool conv = mn == m || u - l <= 2.4e-7f * fabsf(u) + 1e-30f;
            m = mn;
            if (conv) break;
        }
        l1 = mid + half * static_cast<double>(m);
    }
    const double f2v = gp_eval<2>(S.f2, l1), f1v = gp_eval<3>(S.f1, l1), f0v = gp_eval<4>(S.f0, l1);
    const double g1v = gp_eval<1>(S.g1, l1), g0v = gp_eval<2>(S.q, l1);
    double l2;
    const double den = f1v - f2v * g1v;
    if (fabs(den) > 1e-12 * (fabs(f1v) + fabs(f2v * g1v))) {
        l2 = -(f0v - f2v * g0v) / den;
    } else {  // F = f2 G: take the root of G nearer to the vertex (double-root case)
        l2 = -0.5 * g1v + sqrt(fmax(0.25 * g1v * g1v - g0v, 0.0));
    }
    const double Bv = gp_eval<1>(S.B, l1), Cv = gp_eval<1>(S.C, l1), Ev = gp_eval<2>(S.E, l1);
    const double den3 = S.A * l2 + Cv;
    double l3;
    if (fabs(den3) > 1e-12 * (fabs(S.A * l2) + fabs(Cv))) {
        l3 = -(Bv * l2 + Ev) / den3;
    } else {
        const double rv = gp_eval<1>(S.r, l1), sv = gp_eval<2>(S.s, l1);
        l3 = rv + sqrt(fmax(rv * rv - sv, 0.0));
    }
    L[0] = l1;
    L[1] = l2;
    L[2] = l3;
    for (int it = 0; it < 4; ++it) {
        double f[3], J[3][3], dl[3];
        gp_system(o, d, S.D2, L, f, J);
        if (!gp_solve3(J, f, dl)) break;
        L[0] -= dl[0];
        L[1] -= dl[1];
        L[2] -= dl[2];
    }
    double f[3], J[3][3];
    gp_system(o, d, S.D2, L, f, J);
    bool ok = L[0] > 0.0 && L[1] > 0.0 && L[2] > 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) ok = ok && fabs(f[k]) <= 1e-8 * (1.0 + S.D2[k]);
    return ok;
}

// All solutions on one thread (lambda triples, ascending lambda_1, all
// positive; solutions closer than 1e-6 relative are one).
__device__ inline void gp3p_lambdas(const double o[3][3], const double d[3][3], const double X[3][3], Gp3pSol& out) {
    out.n = 0;
    Gp3pSys S;
    if (!gp3p_setup(o, d, X, S)) return;
    Gp3pBracket br[kGp3pMaxSol];
    const int nb = gp3p_brackets(S, br, kGp3pMaxSol);
    for (int i = 0; i < nb; ++i) {
        double L[3];
        bool ok = gp3p_finish(S, o, d, br[i], L);
        for (int j = 0; j < out.n && ok; ++j)
            if (fabs(out.lam[j][0] - L[0]) <= 1e-6 * (1.0 + L[0]) && fabs(out.lam[j][1] - L[1]) <= 1e-6 * (1.0 + L[1]) &&
                fabs(out.lam[j][2] - L[2]) <= 1e-6 * (1.0 + L[2]))
                ok = false;
        if (ok) {
            out.lam[out.n][0] = L[0];
            out.lam[out.n][1] = L[1];
            out.lam[out.n][2] = L[2];
            ++out.n;
        }
    }
}

// orthonormal frame of a triangle: e1 along P1 - P0, e3 normal, e2 = e3 x e1
__device__ __forceinline__ bool gp_frame(const double P0[3], const double P1[3], const double P2[3], double F[3][3]) {
    double u[3], v[3], w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = P1[a] - P0[a];
        v[a] = P2[a] - P0[a];
    }
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
    const double nu = sqrt(dot3d(u, u)), nw = sqrt(dot3d(w, w));
    if (!(nu > 0.0) || !(nw > 0.0)) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        F[0][a] = u[a] / nu;
        F[2][a] = w[a] / nw;
    }
    F[1][0] = F[2][1] * F[0][2] - F[2][2] * F[0][1];
    F[1][1] = F[2][2] * F[0][0] - F[2][0] * F[0][2];
    F[1][2] = F[2][0] * F[0][1] - F[2][1] * F[0][0];
    return true;
}

// rig pose (R, t) with R X_i + t = P_i from the triangles' frames
__device__ __forceinline__ bool gp_pose(const double X[3][3], const double P[3][3], double R[9], double t[3]) {
    double FX[3][3], FP[3][3];
    if (!gp_frame(X[0], X[1], X[2], FX) || !gp_frame(P[0], P[1], P[2], FP)) return false;
    // R = FP^T FX (rows of F are the frame axes)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) R[3 * i + j] = FP[0][i] * FX[0][j] + FP[1][i] * FX[1][j] + FP[2][i] * FX[2][j];
    // t from the centroids
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double cx = (X[0][0] + X[1][0] + X[2][0]) / 3.0, cy = (X[0][1] + X[1][1] + X[2][1]) / 3.0,
                     cz = (X[0][2] + X[1][2] + X[2][2]) / 3.0;
        t[a] = (P[0][a] + P[1][a] + P[2][a]) / 3.0 - (R[3 * a] * cx + R[3 * a + 1] * cy + R[3 * a + 2] * cz);
    }
    return true;
}

}  // namespace imloc
