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
// are not parallel).  The octic is sampled on a grid over that interval with
// Chebyshev spacing (roots crowd towards its ends); each sign change is
// refined by safeguarded Newton, and a cell whose ends agree in sign but not
// in slope is split at the extremum (two close roots).  lambda_2 and
// lambda_3 follow by back-substitution, and Newton on the three distance
// equations polishes the triple.  The pose comes from the two triangles'
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
template <int D>
__device__ __forceinline__ void gp_eval_d(const double (&c)[D + 1], double x, double& p, double& dp) {
    p = c[D];
    dp = 0.0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
        dp = fma(dp, x, p);
        p = fma(p, x, c[k]);
    }
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
// acc += s * a (deg(a) <= deg(acc))
template <int A, int N>
__device__ __forceinline__ void gp_axpy(double (&acc)[N + 1], double s, const double (&a)[A + 1]) {
#pragma unroll
    for (int k = 0; k <= A; ++k) acc[k] = fma(s, a[k], acc[k]);
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

// root of p in [l, u] where p changes sign (p(l) = pl): Newton steps kept
// inside the shrinking bracket, bisection otherwise
__device__ inline double gp_refine(const double (&c)[9], double l, double u, double pl) {
    double x = 0.5 * (l + u);
    for (int it = 0; it < 60; ++it) {
        double px, dpx;
        gp_eval_d<8>(c, x, px, dpx);
        if (px == 0.0) return x;
        if ((px < 0.0) == (pl < 0.0)) {
            l = x;
            pl = px;
        } else {
            u = x;
        }
        double xn = x - px / dpx;
        if (!(xn > l && xn < u)) xn = 0.5 * (l + u);
        const bool conv = fabs(xn - x) <= 1e-15 * fabs(x) || (u - l) <= 1e-15 * fabs(u);
        x = xn;
        if (conv) break;
    }
    return x;
}

// grid point j of kGp3pGrid over [lo, hi] (Chebyshev spacing)
__device__ __forceinline__ double gp_node(int j, double lo, double hi) {
    if (j <= 0) return lo;
    if (j >= kGp3pGrid) return hi;
    return 0.5 * (lo + hi) - 0.5 * (hi - lo) * cospi(static_cast<double>(j) / kGp3pGrid);
}

// The solutions (lambda triples, ascending lambda_1, all positive) whose
// lambda_1 lies in grid cells [cell0, cell1) (all: 0, kGp3pGrid), so that several
// threads can share one minimal sample, each scanning a slice of the grid.
__device__ inline void gp3p_lambdas(const double o[3][3], const double d[3][3], const double X[3][3], Gp3pSol& out,
                                    int cell0 = 0, int cell1 = kGp3pGrid) {
    out.n = 0;
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
    double c[3], a[3], b[3], e[3], D2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = pi[k], j = pj[k];
        double oij[3], x[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            oij[m] = o[i][m] - o[j][m];
            x[m] = X[i][m] - X[j][m];
        }
        D2[k] = dot3d(x, x);
        c[k] = dot3d(d[i], d[j]);
        a[k] = dot3d(d[i], oij);
        b[k] = dot3d(d[j], oij);
        e[k] = dot3d(oij, oij) - D2[k];
    }
    // feasible lambda_1: real lambda_2 (pair 1,2) and real lambda_3 (pair 1,3)
    double lo2, hi2, lo3, hi3;
    if (!gp_feasible(c[0] * c[0] - 1.0, c[0] * b[0] - a[0], b[0] * b[0] - e[0], lo2, hi2)) return;
    if (!gp_feasible(c[1] * c[1] - 1.0, c[1] * b[1] - a[1], b[1] * b[1] - e[1], lo3, hi3)) return;
    double lo = fmax(fmax(lo2, lo3), 0.0), hi = fmin(hi2, hi3);
    if (!(hi > lo)) return;
    const double pad = 1e-9 * (hi - lo) + 1e-12 * hi;
    lo = fmax(lo - pad, 0.0);
    hi += pad;

    // polynomials in lambda_1 (ascending)
    const double p[2] = {b[0], c[0]}, q[3] = {e[0], 2.0 * a[0], 1.0};  // l2^2 - 2 p l2 + q
    const double r[2] = {b[1], c[1]}, s[3] = {e[1], 2.0 * a[1], 1.0};  // l3^2 - 2 r l3 + s
    const double A = -2.0 * c[2];
    const double B[2] = {2.0 * (p[0] + a[2]), 2.0 * p[1]};
    const double C[2] = {2.0 * (r[0] - b[2]), 2.0 * r[1]};
    const double E[3] = {e[2] - q[0] - s[0], -q[1] - s[1], -q[2] - s[2]};
    // F(l2) = f2 l2^2 + f1 l2 + f0 from pair (1,3) with l3 = -(B l2 + E) / (A l2 + C)
    double f2[3], f1[4], f0[5];
    {
        double BB[3], rB[3];
        gp_mul<1, 1>(B, B, BB);
        gp_mul<1, 1>(r, B, rB);
#pragma unroll
        for (int k = 0; k < 3; ++k) f2[k] = BB[k] + 2.0 * A * rB[k] + A * A * s[k];
        double BE[4], BC[3], rBC[4], rE[4], sC[4];
        gp_mul<1, 2>(B, E, BE);
        gp_mul<1, 1>(B, C, BC);
        gp_mul<1, 2>(r, BC, rBC);
        gp_mul<1, 2>(r, E, rE);
        gp_mul<2, 1>(s, C, sC);
#pragma unroll
        for (int k = 0; k < 4; ++k) f1[k] = 2.0 * (BE[k] + rBC[k] + A * rE[k] + A * sC[k]);
        double EE[5], rEC[5], CC[3], sCC[5];
        gp_mul<2, 2>(E, E, EE);
        gp_mul<3, 1>(rE, C, rEC);
        gp_mul<1, 1>(C, C, CC);
        gp_mul<2, 2>(s, CC, sCC);
#pragma unroll
        for (int k = 0; k < 5; ++k) f0[k] = EE[k] + 2.0 * rEC[k] + sCC[k];
    }
    // G(l2) = l2^2 + g1 l2 + g0; resultant (f2 g0 - f0)^2 - (f2 g1 - f1)(f1 g0 - f0 g1)
    const double g1[2] = {-2.0 * p[0], -2.0 * p[1]};
    double oct[9];
    {
        double t1[5], t2[4], t3[6], tmp5[5], tmp4[4], tmp6[6];
        gp_mul<2, 2>(f2, q, tmp5);
#pragma unroll
        for (int k = 0; k < 5; ++k) t1[k] = tmp5[k] - f0[k];
        gp_mul<2, 1>(f2, g1, tmp4);
#pragma unroll
        for (int k = 0; k < 4; ++k) t2[k] = tmp4[k] - f1[k];
        gp_mul<3, 2>(f1, q, tmp6);
#pragma unroll
        for (int k = 0; k < 6; ++k) t3[k] = tmp6[k];
        double f0g1[6];
        gp_mul<4, 1>(f0, g1, f0g1);
#pragma unroll
        for (int k = 0; k < 6; ++k) t3[k] -= f0g1[k];
        double t11[9], t23[9];
        gp_mul<4, 4>(t1, t1, t11);
        gp_mul<3, 5>(t2, t3, t23);
#pragma unroll
        for (int k = 0; k < 9; ++k) oct[k] = t11[k] - t23[k];
    }

    // sign changes of the octic on a grid over [lo, hi], refined by safeguarded
    // Newton.  Two roots closer than the grid step leave no sign change, but p'
    // changes sign between them: such a cell is split at the extremum of p.
    // Chebyshev spacing: roots crowd towards the ends of the feasible interval
    // (where lambda_2 or lambda_3 turns complex), so the cells are finest there
    double xa = gp_node(cell0, lo, hi), pa, dpa;
    gp_eval_d<8>(oct, xa, pa, dpa);
    double roots[kGp3pMaxSol];
    int nroots = 0;
    for (int gi = cell0 + 1; gi <= cell1 && nroots < kGp3pMaxSol; ++gi) {
        const double xb = gp_node(gi, lo, hi);
        double pb, dpb;
        gp_eval_d<8>(oct, xb, pb, dpb);
        if (pa == 0.0) {
            roots[nroots++] = xa;
        } else if (pb != 0.0 && (pa < 0.0) != (pb < 0.0)) {
            roots[nroots++] = gp_refine(oct, xa, xb, pa);
        } else if (pb != 0.0 && (dpa < 0.0) != (dpb < 0.0)) {
            // extremum of p inside the cell: bisection on p'
            double l = xa, u = xb;
            for (int it = 0; it < 50; ++it) {
                const double m = 0.5 * (l + u);
                double pm, dpm;
                gp_eval_d<8>(oct, m, pm, dpm);
                if ((dpm < 0.0) == (dpa < 0.0)) l = m; else u = m;
            }
            const double xe = 0.5 * (l + u);
            const double pe = gp_eval<8>(oct, xe);
            if ((pe < 0.0) != (pa < 0.0) && nroots + 2 <= kGp3pMaxSol) {
                roots[nroots++] = gp_refine(oct, xa, xe, pa);
                roots[nroots++] = gp_refine(oct, xe, xb, pe);
            }
        }
        xa = xb;
        pa = pb;
        dpa = dpb;
    }

    for (int ri = 0; ri < nroots; ++ri) {
        // back-substitution: the common root of F and G, then l3 from the bilinear relation
        const double l1 = roots[ri];
        const double f2v = gp_eval<2>(f2, l1), f1v = gp_eval<3>(f1, l1), f0v = gp_eval<4>(f0, l1);
        const double g1v = gp_eval<1>(g1, l1), g0v = gp_eval<2>(q, l1);
        double l2;
        const double den = f1v - f2v * g1v;
        if (fabs(den) > 1e-12 * (fabs(f1v) + fabs(f2v * g1v))) {
            l2 = -(f0v - f2v * g0v) / den;
        } else {  // F = f2 G: take the root of G nearer to the vertex (double-root case)
            l2 = -0.5 * g1v + sqrt(fmax(0.25 * g1v * g1v - g0v, 0.0));
        }
        const double Bv = gp_eval<1>(B, l1), Cv = gp_eval<1>(C, l1), Ev = gp_eval<2>(E, l1);
        const double den3 = A * l2 + Cv;
        double l3;
        if (fabs(den3) > 1e-12 * (fabs(A * l2) + fabs(Cv))) {
            l3 = -(Bv * l2 + Ev) / den3;
        } else {
            const double rv = gp_eval<1>(r, l1), sv = gp_eval<2>(s, l1);
            l3 = rv + sqrt(fmax(rv * rv - sv, 0.0));
        }
        double L[3] = {l1, l2, l3};
        for (int it = 0; it < 4; ++it) {
            double f[3], J[3][3], dl[3];
            gp_system(o, d, D2, L, f, J);
            if (!gp_solve3(J, f, dl)) break;
            L[0] -= dl[0];
            L[1] -= dl[1];
            L[2] -= dl[2];
        }
        double f[3], J[3][3];
        gp_system(o, d, D2, L, f, J);
        bool ok = L[0] > 0.0 && L[1] > 0.0 && L[2] > 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) ok = ok && fabs(f[k]) <= 1e-8 * (1.0 + D2[k]);
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
