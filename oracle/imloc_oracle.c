/*
 * imloc_oracle.c -- plain FP64 CPU oracle of the ImLoc localization hot path
 * (lift + LO-RANSAC PnP, ImLoc Sec. 3.3).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  Written for
 * reading, not speed: every step follows the definition in the order the
 * paper states it, in double precision, one query on one thread.  Decisions
 * that the paper leaves open are the readings listed in the design notes
 * (pixel centres at +0.5, z-depth, reject-on-invalid-tap, deterministic
 * stride subsampling, Philox counter layout, round-level LO trigger, LO and
 * Cauchy refinement schedules).
 */
#include "imloc_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ======================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, with a   */
/* Weyl-sequence key schedule.                                                */
/* ======================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = (uint64_t)mult0 * c[0];
        uint64_t p1 = (uint64_t)mult1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* ======================================================================== */
/* Lift (Sec. 3.3, "Query Time Matching and 2D-3D Lifting"): keep a match    */
/* whose confidence exceeds 0.05 and whose depth is valid; query->database   */
/* matches take the bilinear depth at the subpixel database position,        */
/* database->query matches look the depth up; back-project through the      */
/* database intrinsics and pose into the world.                              */
/* ======================================================================== */
static int depth_ok(float d) { return isfinite(d) && d > 0.0f; }

int64_t orc_lift(const orc_view* views, int64_t n_views,
                 const float* q_u, const float* q_v, const float* db_u, const float* db_v,
                 const float* conf, const int64_t* seg_off, const int32_t* seg_view,
                 const int32_t* seg_dir, int64_t n_seg, float conf_min,
                 double* out_x, double* out_y, double* out_X, double* out_w, int64_t* out_src)
{
    int64_t n_out = 0;
    for (int64_t s = 0; s < n_seg; ++s) {
        if (seg_view[s] < 0 || seg_view[s] >= n_views) continue;
        const orc_view* v = &views[seg_view[s]];
        for (int64_t i = seg_off[s]; i < seg_off[s + 1]; ++i) {
            /* the threshold decision is taken in the precision of the input (float) */
            if (!(conf[i] > conf_min)) continue;
            double u = db_u[i], vv = db_v[i];
            if (!isfinite(u) || !isfinite(vv)) continue;
            double d;
            if (seg_dir[s] == 0) {
                /* bilinear between the four surrounding pixel centres */
                double a = u - 0.5, b = vv - 0.5;
                double fa = floor(a), fb = floor(b);
                if (fa < 0.0 || fa + 1.0 > (double)(v->width - 1)) continue;
                if (fb < 0.0 || fb + 1.0 > (double)(v->height - 1)) continue;
                int64_t i0 = (int64_t)fa, j0 = (int64_t)fb;
                float d00 = v->depth[j0 * v->pitch + i0];
                float d01 = v->depth[j0 * v->pitch + i0 + 1];
                float d10 = v->depth[(j0 + 1) * v->pitch + i0];
                float d11 = v->depth[(j0 + 1) * v->pitch + i0 + 1];
                if (!depth_ok(d00) || !depth_ok(d01) || !depth_ok(d10) || !depth_ok(d11)) continue;
                double al = a - fa, be = b - fb;
                d = (1.0 - be) * ((1.0 - al) * d00 + al * d01) + be * ((1.0 - al) * d10 + al * d11);
            } else {
                double fa = floor(u), fb = floor(vv);
                if (fa < 0.0 || fa > (double)(v->width - 1)) continue;
                if (fb < 0.0 || fb > (double)(v->height - 1)) continue;
                float dd = v->depth[(int64_t)fb * v->pitch + (int64_t)fa];
                if (!depth_ok(dd)) continue;
                d = dd;
            }
            /* z-depth: the camera-frame point is d * K^-1 [u, v, 1]^T */
            double Xc[3] = {d * (u - v->cx) / v->fx, d * (vv - v->cy) / v->fy, d};
            double D[3] = {Xc[0] - v->t[0], Xc[1] - v->t[1], Xc[2] - v->t[2]};
            /* X_w = R^T (X_c - t) */
            for (int r = 0; r < 3; ++r)
                out_X[3 * n_out + r] = v->R[0 * 3 + r] * D[0] + v->R[1 * 3 + r] * D[1] + v->R[2 * 3 + r] * D[2];
            out_x[n_out] = q_u[i];
            out_y[n_out] = q_v[i];
            out_w[n_out] = conf[i];
            out_src[n_out] = i;
            ++n_out;
        }
    }
    return n_out;
}

/* ======================================================================== */
/* Uniform subsampling to at most m scoring correspondences (Sec. 3.3):      */
/* deterministic stride idx_k = floor(k n / m).                              */
/* ======================================================================== */
void orc_subsample(int64_t n, int64_t m, int64_t* idx)
{
    for (int64_t k = 0; k < m; ++k) idx[k] = (int64_t)(((__int128)k * n) / m);
}

/* ======================================================================== */
/* Minimal sample: key = seed, counter = (sample, query, attempt, 0); the    */
/* first three outputs map to [0,m) by the high word of r*m.                 */
/* ======================================================================== */
int orc_sample(uint64_t seed, uint32_t query_id, uint32_t sample_id, int64_t m, int64_t out[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t attempt = 0; attempt < 16; ++attempt) {
        uint32_t ctr[4] = {sample_id, query_id, attempt, 0u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        for (int k = 0; k < 3; ++k) out[k] = (int64_t)(((uint64_t)r[k] * (uint64_t)m) >> 32);
        if (out[0] != out[1] && out[0] != out[2] && out[1] != out[2]) return (int)attempt;
    }
    return -1;
}

/* ======================================================================== */
/* P3P.  Independent formulation from the GPU path: Grunert's substitution   */
/* lambda2 = u lambda1, lambda3 = v lambda1 turns the three distance         */
/* equations into two conics in (u, v); their resultant in u is a quartic in */
/* v whose real roots are found as polynomial roots (Durand-Kerner + Newton  */
/* polish).  The pose follows from the three camera-frame points by Horn's   */
/* closed-form absolute orientation (unit quaternion, 4x4 eigenvector).      */
/* ======================================================================== */
static void poly_mul(const double* a, int da, const double* b, int db, double* out)
{
    for (int k = 0; k <= da + db; ++k) out[k] = 0.0;
    for (int i = 0; i <= da; ++i)
        for (int j = 0; j <= db; ++j) out[i + j] += a[i] * b[j];
}

static double poly_eval(const double* c, int deg, double x)
{
    double acc = 0.0;
    for (int k = deg; k >= 0; --k) acc = acc * x + c[k];
    return acc;
}

static double poly_deriv_eval(const double* c, int deg, double x)
{
    double acc = 0.0;
    for (int k = deg; k >= 1; --k) acc = acc * x + k * c[k];
    return acc;
}

/* real roots of sum_k c[k] x^k (deg <= 4); returns the count */
static int poly_real_roots(const double* c_in, int deg, double* roots)
{
    double c[5];
    double cmax = 0.0;
    for (int k = 0; k <= deg; ++k) { c[k] = c_in[k]; cmax = fmax(cmax, fabs(c[k])); }
    if (cmax == 0.0) return 0;
    while (deg > 0 && fabs(c[deg]) <= 1e-14 * cmax) --deg;
    if (deg == 0) return 0;
    if (deg == 1) { roots[0] = -c[0] / c[1]; return 1; }
    double complex z[4];
    double a[5];
    for (int k = 0; k <= deg; ++k) a[k] = c[k] / c[deg];
    double bound = 1.0;
    for (int k = 0; k < deg; ++k) bound = fmax(bound, 1.0 + fabs(a[k]));
    double complex seed = 0.4 + 0.9 * I;
    double complex p = 1.0;
    for (int k = 0; k < deg; ++k) { p *= seed; z[k] = p * (0.5 * bound); }
    for (int it = 0; it < 2000; ++it) {
        double change = 0.0;
        for (int k = 0; k < deg; ++k) {
            double complex num = 0.0;
            for (int j = deg; j >= 0; --j) num = num * z[k] + a[j];
            double complex den = 1.0;
            for (int j = 0; j < deg; ++j)
                if (j != k) den *= (z[k] - z[j]);
            if (cabs(den) == 0.0) den = 1e-300;
            double complex dz = num / den;
            z[k] -= dz;
            change = fmax(change, cabs(dz) / (1.0 + cabs(z[k])));
        }
        if (change < 1e-16) break;
    }
    int nr = 0;
    for (int k = 0; k < deg; ++k) {
        if (fabs(cimag(z[k])) > 1e-6 * (1.0 + cabs(z[k]))) continue;
        double x = creal(z[k]);
        for (int it = 0; it < 8; ++it) {
            double d = poly_deriv_eval(c, deg, x);
            if (d == 0.0) break;
            double step = poly_eval(c, deg, x) / d;
            x -= step;
            if (fabs(step) <= 1e-17 * (1.0 + fabs(x))) break;
        }
        int dup = 0;
        for (int j = 0; j < nr; ++j)
            if (fabs(roots[j] - x) <= 1e-10 * (1.0 + fabs(x))) dup = 1;
        if (!dup) roots[nr++] = x;
    }
    return nr;
}

/* eigenvector of the largest eigenvalue of a symmetric 4x4 (cyclic Jacobi) */
static void sym4_top_eigvec(const double Ain[16], double v_out[4])
{
    double A[4][4], V[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) { A[i][j] = Ain[4 * i + j]; V[i][j] = (i == j) ? 1.0 : 0.0; }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                tot += A[i][j] * A[i][j];
                if (i != j) off += A[i][j] * A[i][j];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(tt * tt + 1.0), sn = tt * cs;
                for (int k = 0; k < 4; ++k) { /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 4; ++k) { /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (A[i][i] > A[best][best]) best = i;
    for (int k = 0; k < 4; ++k) v_out[k] = V[k][best];
}

/* Horn (1987): rotation R and translation t with C_i = R X_i + t */
static void horn_absolute_orientation(const double Xw[9], const double Xc[9], double R[9], double t[3])
{
    double mw[3] = {0, 0, 0}, mc[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) { mw[a] += Xw[3 * i + a] / 3.0; mc[a] += Xc[3 * i + a] / 3.0; }
    double S[3][3] = {{0}};
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) S[a][b] += (Xw[3 * i + a] - mw[a]) * (Xc[3 * i + b] - mc[b]);
    double Sxx = S[0][0], Sxy = S[0][1], Sxz = S[0][2];
    double Syx = S[1][0], Syy = S[1][1], Syz = S[1][2];
    double Szx = S[2][0], Szy = S[2][1], Szz = S[2][2];
    double N[16] = {
        Sxx + Syy + Szz, Syz - Szy,        Szx - Sxz,        Sxy - Syx,
        Syz - Szy,       Sxx - Syy - Szz,  Sxy + Syx,        Szx + Sxz,
        Szx - Sxz,       Sxy + Syx,        -Sxx + Syy - Szz, Syz + Szy,
        Sxy - Syx,       Szx + Sxz,        Syz + Szy,        -Sxx - Syy + Szz};
    double q[4];
    sym4_top_eigvec(N, q);
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double nq = sqrt(w * w + x * x + y * y + z * z);
    w /= nq; x /= nq; y /= nq; z /= nq;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    for (int a = 0; a < 3; ++a) t[a] = mc[a] - (R[3 * a] * mw[0] + R[3 * a + 1] * mw[1] + R[3 * a + 2] * mw[2]);
}

/* residuals of the three distance equations lambda_i^2 + lambda_j^2 - 2 b_ij lambda_i lambda_j = a_ij */
static void p3p_residual(const double L[3], const double a[3], const double b[3], double f[3])
{
    f[0] = L[0] * L[0] + L[1] * L[1] - 2 * b[0] * L[0] * L[1] - a[0];
    f[1] = L[0] * L[0] + L[2] * L[2] - 2 * b[1] * L[0] * L[2] - a[1];
    f[2] = L[1] * L[1] + L[2] * L[2] - 2 * b[2] * L[1] * L[2] - a[2];
}

static int solve3(double A[3][3], const double b[3], double x[3])
{
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (det == 0.0 || !isfinite(det)) return 0;
    for (int c = 0; c < 3; ++c) {
        double M[3][3];
        memcpy(M, A, sizeof(M));
        for (int r = 0; r < 3; ++r) M[r][c] = b[r];
        x[c] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
              - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
              + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
    }
    return 1;
}

int orc_p3p(const double y[9], const double X[9], double R_out[36], double t_out[12], double lambda_out[12])
{
    double a12 = 0, a13 = 0, a23 = 0;
    for (int k = 0; k < 3; ++k) {
        a12 += (X[k] - X[3 + k]) * (X[k] - X[3 + k]);
        a13 += (X[k] - X[6 + k]) * (X[k] - X[6 + k]);
        a23 += (X[3 + k] - X[6 + k]) * (X[3 + k] - X[6 + k]);
    }
    double b12 = y[0] * y[3] + y[1] * y[4] + y[2] * y[5];
    double b13 = y[0] * y[6] + y[1] * y[7] + y[2] * y[8];
    double b23 = y[3] * y[6] + y[4] * y[7] + y[5] * y[8];
    if (!(a12 > 0) || !(a13 > 0) || !(a23 > 0)) return 0;

    /* With lambda2 = u lambda1 and lambda3 = v lambda1 the ratios of the
     * distance equations give two quadratics in u whose coefficients are
     * polynomials in v:
     *   P(u) = a13 (1 + u^2 - 2 b12 u) - a12 (1 + v^2 - 2 b13 v)
     *   Q(u) = a23 (1 + u^2 - 2 b12 u) - a12 (u^2 + v^2 - 2 b23 u v)    */
    double p2 = a13, p1 = -2.0 * a13 * b12;
    double p0[3] = {a13 - a12, 2.0 * a12 * b13, -a12};
    double q2 = a23 - a12;
    double q1[2] = {-2.0 * a23 * b12, 2.0 * a12 * b23};
    double q0[3] = {a23, 0.0, -a12};
    /* Resultant of two quadratics: (p2 q0 - q2 p0)^2 - (p2 q1 - q2 p1)(p1 q0 - q1 p0) */
    double A[3], Bv[2], C[4], A2[5], BC[5], res[5];
    for (int k = 0; k < 3; ++k) A[k] = p2 * q0[k] - q2 * p0[k];
    Bv[0] = p2 * q1[0] - q2 * p1;
    Bv[1] = p2 * q1[1];
    double q1p0[4];
    poly_mul(q1, 1, p0, 2, q1p0);
    for (int k = 0; k < 4; ++k) C[k] = (k < 3 ? p1 * q0[k] : 0.0) - q1p0[k];
    poly_mul(A, 2, A, 2, A2);
    poly_mul(Bv, 1, C, 3, BC);
    for (int k = 0; k < 5; ++k) res[k] = A2[k] - BC[k];

    double vr[4];
    int nv = poly_real_roots(res, 4, vr);
    double sol_L[4][3];
    int ns = 0;
    const double av[3] = {a12, a13, a23}, bv[3] = {b12, b13, b23};
    for (int k = 0; k < nv; ++k) {
        double v = vr[k];
        double den = -(Bv[0] + Bv[1] * v); /* q2 p1 - p2 q1(v) */
        double num = A[0] + A[1] * v + A[2] * v * v;
        if (fabs(den) <= 1e-14 * (fabs(num) + 1e-300)) continue;
        double u = num / den;
        double s = 1.0 + v * v - 2.0 * b13 * v;
        if (!(s > 0)) continue;
        double L[3];
        L[0] = sqrt(a13 / s);
        L[1] = u * L[0];
        L[2] = v * L[0];
        /* Newton polish on the three distance equations */
        for (int it = 0; it < 4; ++it) {
            double f[3];
            p3p_residual(L, av, bv, f);
            double J[3][3] = {
                {2 * L[0] - 2 * b12 * L[1], 2 * L[1] - 2 * b12 * L[0], 0},
                {2 * L[0] - 2 * b13 * L[2], 0, 2 * L[2] - 2 * b13 * L[0]},
                {0, 2 * L[1] - 2 * b23 * L[2], 2 * L[2] - 2 * b23 * L[1]}};
            double dl[3];
            if (!solve3(J, f, dl)) break;
            for (int a = 0; a < 3; ++a) L[a] -= dl[a];
        }
        if (!(L[0] > 0 && L[1] > 0 && L[2] > 0)) continue;
        double f[3];
        p3p_residual(L, av, bv, f);
        if (fabs(f[0]) > 1e-8 * a12 || fabs(f[1]) > 1e-8 * a13 || fabs(f[2]) > 1e-8 * a23) continue;
        int dup = 0;
        for (int j = 0; j < ns; ++j)
            if (fabs(sol_L[j][0] - L[0]) <= 1e-9 * L[0] && fabs(sol_L[j][1] - L[1]) <= 1e-9 * L[1] &&
                fabs(sol_L[j][2] - L[2]) <= 1e-9 * L[2])
                dup = 1;
        if (dup) continue;
        memcpy(sol_L[ns++], L, sizeof(L));
    }
    /* canonical order: ascending depth of the first point */
    for (int i = 1; i < ns; ++i)
        for (int j = i; j > 0 && sol_L[j][0] < sol_L[j - 1][0]; --j) {
            double tmp[3];
            memcpy(tmp, sol_L[j], sizeof(tmp));
            memcpy(sol_L[j], sol_L[j - 1], sizeof(tmp));
            memcpy(sol_L[j - 1], tmp, sizeof(tmp));
        }
    for (int k = 0; k < ns; ++k) {
        double Xc[9];
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 3; ++a) Xc[3 * i + a] = sol_L[k][i] * y[3 * i + a];
        horn_absolute_orientation(X, Xc, &R_out[9 * k], &t_out[3 * k]);
        if (lambda_out)
            for (int i = 0; i < 3; ++i) lambda_out[3 * k + i] = sol_L[k][i];
    }
    return ns;
}

/* ======================================================================== */
/* Scoring: confidence-weighted truncated squared reprojection error (MSAC). */
/* A point behind the camera (Z <= 0) counts as an outlier.                  */
/* ======================================================================== */
static int project_residual(const orc_corr* c, int64_t i, const orc_cam* cam, const double R[9],
                            const double t[3], double Xc[3], double r[2])
{
    const double* Xw = &c->X[3 * i];
    for (int a = 0; a < 3; ++a) Xc[a] = R[3 * a] * Xw[0] + R[3 * a + 1] * Xw[1] + R[3 * a + 2] * Xw[2] + t[a];
    if (!(Xc[2] > 0.0)) return 0;
    r[0] = cam->fx * Xc[0] / Xc[2] + cam->cx - c->x[i];
    r[1] = cam->fy * Xc[1] / Xc[2] + cam->cy - c->y[i];
    return 1;
}

double orc_score(const orc_corr* c, const int64_t* idx, int64_t m, const orc_cam* cam,
                 const double R[9], const double t[3], double tau, int64_t* inliers)
{
    double tau2 = tau * tau, s = 0.0;
    int64_t cnt = 0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double Xc[3], r[2];
        double r2 = tau2;
        if (project_residual(c, i, cam, R, t, Xc, r)) {
            r2 = r[0] * r[0] + r[1] * r[1];
            if (r2 < tau2) ++cnt;
        }
        s += c->w[i] * (r2 < tau2 ? r2 : tau2);
    }
    if (inliers) *inliers = cnt;
    return s;
}

/* ======================================================================== */
/* Gauss-Newton on SE(3) with a left perturbation X_c' = Exp(w) X_c + v.     */
/* ======================================================================== */
static void jacobian(const double Xc[3], const orc_cam* cam, double J[2][6])
{
    double X = Xc[0], Y = Xc[1], Z = Xc[2];
    double du[3] = {cam->fx / Z, 0.0, -cam->fx * X / (Z * Z)};
    double dv[3] = {0.0, cam->fy / Z, -cam->fy * Y / (Z * Z)};
    /* d X_c' / d w = -[X_c]_x */
    double M[3][3] = {{0.0, Z, -Y}, {-Z, 0.0, X}, {Y, -X, 0.0}};
    for (int k = 0; k < 3; ++k) {
        J[0][k] = du[0] * M[0][k] + du[1] * M[1][k] + du[2] * M[2][k];
        J[1][k] = dv[0] * M[0][k] + dv[1] * M[1][k] + dv[2] * M[2][k];
        J[0][3 + k] = du[k];
        J[1][3 + k] = dv[k];
    }
}

static void so3_exp(const double w[3], double E[9])
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double A, B;
    if (th < 1e-8) { A = 1.0 - th2 / 6.0; B = 0.5 - th2 / 24.0; }
    else { A = sin(th) / th; B = (1.0 - cos(th)) / th2; }
    double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double K2 = 0;
            for (int k = 0; k < 3; ++k) K2 += K[3 * i + k] * K[3 * k + j];
            E[3 * i + j] = (i == j ? 1.0 : 0.0) + A * K[3 * i + j] + B * K2;
        }
}

static void apply_update(const double d[6], const double R[9], const double t[3], double Rn[9], double tn[3])
{
    double E[9];
    so3_exp(d, E);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            Rn[3 * i + j] = E[3 * i] * R[j] + E[3 * i + 1] * R[3 + j] + E[3 * i + 2] * R[6 + j];
        tn[i] = E[3 * i] * t[0] + E[3 * i + 1] * t[1] + E[3 * i + 2] * t[2] + d[3 + i];
    }
}

static int cholesky_solve6(const double H[36], const double g[6], double x[6])
{
    double L[36] = {0};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = H[6 * i + j];
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[6 * i + i] = sqrt(s);
            } else {
                L[6 * i + j] = s / L[6 * j + j];
            }
        }
    double z[6];
    for (int i = 0; i < 6; ++i) {
        double s = g[i];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * z[k];
        z[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = z[i];
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
    return 1;
}

enum { LOSS_TRUNCATED = 0, LOSS_CAUCHY = 1 };

static double robust_cost(const orc_corr* c, const int64_t* idx, int64_t m, const orc_cam* cam,
                          int loss, double tau, double cs, const double R[9], const double t[3])
{
    double tau2 = tau * tau, cs2 = cs * cs, s = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double Xc[3], r[2], r2 = tau2;
        if (project_residual(c, i, cam, R, t, Xc, r)) r2 = r[0] * r[0] + r[1] * r[1];
        if (loss == LOSS_TRUNCATED) s += c->w[i] * (r2 < tau2 ? r2 : tau2);
        else s += c->w[i] * cs2 * log1p(r2 / cs2);
    }
    return s;
}

/* Returns the number of accepted steps; R, t updated in place; *cost_io holds the cost. */
static int gauss_newton(const orc_corr* c, const int64_t* idx, int64_t m, const orc_cam* cam, int loss,
                        double tau, double cs, int64_t iters, double R[9], double t[3], double* cost_io)
{
    double tau2 = tau * tau, cs2 = cs * cs;
    double cost = robust_cost(c, idx, m, cam, loss, tau, cs, R, t);
    int accepted_steps = 0;
    for (int64_t it = 0; it < iters; ++it) {
        double H[36] = {0}, g[6] = {0};
        int64_t used = 0;
        for (int64_t k = 0; k < m; ++k) {
            int64_t i = idx ? idx[k] : k;
            double Xc[3], r[2];
            if (!project_residual(c, i, cam, R, t, Xc, r)) continue;
            double r2 = r[0] * r[0] + r[1] * r[1];
            double wt;
            if (loss == LOSS_TRUNCATED) {
                if (!(r2 < tau2)) continue; /* outliers sit on the flat part of the loss */
                wt = c->w[i];
            } else {
                wt = c->w[i] / (1.0 + r2 / cs2); /* IRLS weight of the Cauchy loss */
            }
            double J[2][6];
            jacobian(Xc, cam, J);
            for (int a = 0; a < 6; ++a) {
                g[a] += wt * (J[0][a] * r[0] + J[1][a] * r[1]);
                for (int b = 0; b < 6; ++b) H[6 * a + b] += wt * (J[0][a] * J[0][b] + J[1][a] * J[1][b]);
            }
            ++used;
        }
        if (used < 3) break;
        double mu = 0.0;
        int ok = 0;
        double d[6], Rn[9], tn[3], cn = cost;
        for (int attempt = 0; attempt < 4; ++attempt) {
            double Hd[36], mg[6];
            memcpy(Hd, H, sizeof(Hd));
            for (int a = 0; a < 6; ++a) { Hd[7 * a] += mu * H[7 * a]; mg[a] = -g[a]; }
            if (cholesky_solve6(Hd, mg, d)) {
                apply_update(d, R, t, Rn, tn);
                cn = robust_cost(c, idx, m, cam, loss, tau, cs, Rn, tn);
                if (cn < cost) { ok = 1; break; }
            }
            mu = (mu == 0.0) ? 1e-3 : mu * 10.0;
        }
        if (!ok) break;
        const double decrease = cost - cn;
        memcpy(R, Rn, sizeof(Rn));
        memcpy(t, tn, sizeof(tn));
        ++accepted_steps;
        double dn = 0;
        for (int a = 0; a < 6; ++a) dn += d[a] * d[a];
        /* converged: a tiny step, or a step that lowered the cost by < 1e-6 of it */
        const int converged = sqrt(dn) < 1e-10 || decrease < 1e-6 * cost;
        cost = cn;
        if (converged) break;
    }
    *cost_io = cost;
    return accepted_steps;
}

double orc_lo(const orc_corr* c, const int64_t* idx, int64_t m, const orc_cam* cam, double tau,
              int64_t iters, double R[9], double t[3])
{
    double cost;
    gauss_newton(c, idx, m, cam, LOSS_TRUNCATED, tau, 1.0, iters, R, t, &cost);
    return cost;
}

int orc_refine(const orc_corr* c, const int64_t* sel, int64_t n_sel, const orc_cam* cam, double cauchy_c,
               double tau, int64_t iters, double R[9], double t[3])
{
    double cost;
    return gauss_newton(c, sel, n_sel, cam, LOSS_CAUCHY, tau, cauchy_c, iters, R, t, &cost);
}

/* ======================================================================== */
/* Adaptive stop: the chance that none of k minimal sets of 3 is all-inlier  */
/* is (1 - eps^3)^k; stop once it falls below p_miss.                        */
/* ======================================================================== */
double orc_needed_iters(double eps, double p_miss)
{
    double e3 = eps * eps * eps;
    if (e3 >= 1.0) return 0.0;
    if (e3 <= 0.0) return INFINITY;
    return log(p_miss) / log(1.0 - e3);
}

/* ======================================================================== */
/* The LO-RANSAC loop (Sec. 3.3): rounds of `batch` minimal sets; score      */
/* every P3P pose of the round on the subset; if the round's best beats the  */
/* global best, run LO on it; stop at max_iters or by the adaptive rule;     */
/* refine on all inliers of the full set with the Cauchy loss.               */
/* ======================================================================== */
static void bearing(const orc_corr* c, int64_t i, const orc_cam* cam, double out[3])
{
    double b[3] = {(c->x[i] - cam->cx) / cam->fx, (c->y[i] - cam->cy) / cam->fy, 1.0};
    double n = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    for (int a = 0; a < 3; ++a) out[a] = b[a] / n;
}

int orc_ransac_pnp(const orc_corr* c, const orc_cam* cam, const orc_opts* o, orc_result* res,
                   uint8_t* inlier_mask, int64_t* round_best_id, double* round_best_score, int64_t max_rounds)
{
    memset(res, 0, sizeof(*res));
    res->best_hyp = -1;
    int64_t n = c->n;
    if (n < 3) { res->status = -1; return -1; }
    int64_t m = n < o->max_score_corr ? n : o->max_score_corr;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    orc_subsample(n, m, idx);

    int64_t total, batch;
    int64_t (*triples)[3] = NULL;
    if (o->enumerate_all) {
        total = m * (m - 1) * (m - 2) / 6;
        triples = malloc(sizeof(*triples) * (size_t)(total > 0 ? total : 1));
        int64_t s = 0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = i + 1; j < m; ++j)
                for (int64_t k = j + 1; k < m; ++k) { triples[s][0] = i; triples[s][1] = j; triples[s][2] = k; ++s; }
        batch = total > 0 ? total : 1;
    } else {
        total = o->max_iters;
        batch = o->batch;
    }

    double best_R[9], best_t[3], best_score = INFINITY;
    int have_best = 0;
    int64_t subset_inliers = 0, hyps = 0, rounds = 0, iters = 0;
    for (int64_t r = 0;; ++r) {
        int64_t s0 = r * batch, s1 = s0 + batch < total ? s0 + batch : total;
        if (s0 >= total) break;
        double rb_score = INFINITY, rb_R[9], rb_t[3];
        int64_t rb_id = -1;
        for (int64_t s = s0; s < s1; ++s) {
            int64_t tri[3];
            if (triples) memcpy(tri, triples[s], sizeof(tri));
            else if (orc_sample(o->seed, o->query_id, (uint32_t)s, m, tri) < 0) continue;
            double y[9], X[9];
            for (int k = 0; k < 3; ++k) {
                int64_t i = idx[tri[k]];
                bearing(c, i, cam, &y[3 * k]);
                for (int a = 0; a < 3; ++a) X[3 * k + a] = c->X[3 * i + a];
            }
            double Rs[36], ts[12];
            int ns = orc_p3p(y, X, Rs, ts, NULL);
            for (int k = 0; k < ns; ++k) {
                double sc = orc_score(c, idx, m, cam, &Rs[9 * k], &ts[3 * k], o->tau, NULL);
                ++hyps;
                if (sc < rb_score) { /* ascending ids: a tie keeps the lower id */
                    rb_score = sc;
                    rb_id = 4 * s + k;
                    memcpy(rb_R, &Rs[9 * k], sizeof(rb_R));
                    memcpy(rb_t, &ts[3 * k], sizeof(rb_t));
                }
            }
        }
        if (r < max_rounds) {
            if (round_best_id) round_best_id[r] = rb_id;
            if (round_best_score) round_best_score[r] = rb_score;
        }
        if (rb_id >= 0 && rb_score < best_score) {
            memcpy(best_R, rb_R, sizeof(rb_R));
            memcpy(best_t, rb_t, sizeof(rb_t));
            best_score = rb_score;
            res->best_hyp = rb_id;
            have_best = 1;
            if (o->lo_enabled) {
                double lR[9], lt[3];
                memcpy(lR, best_R, sizeof(lR));
                memcpy(lt, best_t, sizeof(lt));
                double ls = orc_lo(c, idx, m, cam, o->tau, o->lo_iters, lR, lt);
                res->lo_count++;
                if (ls < best_score) {
                    memcpy(best_R, lR, sizeof(lR));
                    memcpy(best_t, lt, sizeof(lt));
                    best_score = ls;
                }
            }
            orc_score(c, idx, m, cam, best_R, best_t, o->tau, &subset_inliers);
        }
        iters = s1;
        rounds = r + 1;
        if (iters >= total) break;
        if (o->p_miss > 0.0 && have_best &&
            (double)iters >= orc_needed_iters((double)subset_inliers / (double)m, o->p_miss))
            break;
    }
    free(triples);
    res->iterations = iters;
    res->rounds = rounds;
    res->hypotheses = hyps;
    if (!have_best) { free(idx); res->status = -1; return -1; }
    memcpy(res->R_best, best_R, sizeof(best_R));
    memcpy(res->t_best, best_t, sizeof(best_t));
    res->score = best_score;
    res->subset_inliers = subset_inliers;

    double R[9], t[3];
    memcpy(R, best_R, sizeof(R));
    memcpy(t, best_t, sizeof(t));
    if (o->final_enabled) {
        int64_t* sel = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        int64_t ns = 0;
        double tau2 = o->tau * o->tau;
        for (int64_t i = 0; i < n; ++i) {
            double Xc[3], rr[2];
            if (project_residual(c, i, cam, R, t, Xc, rr) && rr[0] * rr[0] + rr[1] * rr[1] < tau2) sel[ns++] = i;
        }
        orc_refine(c, sel, ns, cam, o->cauchy_scale, o->tau, o->final_iters, R, t);
        free(sel);
    }
    memcpy(res->R, R, sizeof(R));
    memcpy(res->t, t, sizeof(t));
    int64_t cnt = 0;
    double tau2 = o->tau * o->tau;
    for (int64_t i = 0; i < n; ++i) {
        double Xc[3], rr[2];
        int in = project_residual(c, i, cam, R, t, Xc, rr) && rr[0] * rr[0] + rr[1] * rr[1] < tau2;
        if (inlier_mask) inlier_mask[i] = (uint8_t)in;
        cnt += in;
    }
    res->num_inliers = cnt;
    free(idx);
    res->status = 0;
    return 0;
}

/* ==========================================================================
 * Depth codec -- Sec. 3.3 "Data Compression" (clip to [0.25, 128] m, log
 * space, 256 levels) and Sec. 4.3 "Depth Quantization" (8 bits, < 1.4 %
 * relative error).  Reading: code 0 marks a pixel without depth (the mapping
 * keeps only depths with enough support), codes 1..255 are the 255 log-
 * uniform levels from 0.25 m to 128 m; nearest level in log space.
 * ========================================================================== */
double orc_depth_decode_log8(uint8_t code)
{
    if (code == 0) return 0.0;
    return 0.25 * pow(512.0, (double)(code - 1) / 254.0);
}

uint8_t orc_depth_encode_log8(float depth)
{
    if (!isfinite(depth) || !(depth > 0.0f)) return 0;
    double d = (double)depth;
    if (d < 0.25) d = 0.25;
    if (d > 128.0) d = 128.0;
    /* position on the level grid: 0 at 0.25 m, 254 at 128 m */
    const double pos = 254.0 * log(d / 0.25) / log(512.0);
    long level = (long)floor(pos + 0.5);
    if (level < 0) level = 0;
    if (level > 254) level = 254;
    return (uint8_t)(level + 1);
}

void orc_depth_encode_log8_n(const float* depth, int64_t n, uint8_t* codes)
{
    for (int64_t i = 0; i < n; ++i) codes[i] = orc_depth_encode_log8(depth[i]);
}

void orc_depth_decode_log8_n(const uint8_t* codes, int64_t n, double* depth)
{
    for (int64_t i = 0; i < n; ++i) depth[i] = orc_depth_decode_log8(codes[i]);
}

/* ==========================================================================
 * Dense triangulation -- Sec. 3.3 "Depth Estimation by Dense Matching".
 * Readings (the paper does not spell them out): a match's depth hypothesis
 * is where the reference ray passes closest to the match's source ray; the
 * angular error of a match at a point is the angle between the source ray
 * and the direction from the source centre to the point; ties between
 * hypotheses go to the lowest source index; the refinement starts at the
 * winning hypothesis and keeps its inlier set.
 * ========================================================================== */
static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

double orc_angle(const double a[3], const double b[3])
{
    double c[3];
    cross3(a, b, c);
    return atan2(sqrt(dot3(c, c)), dot3(a, b));
}

double orc_closest_depth(const double C0[3], const double d0[3], const double C1[3], const double d1[3])
{
    /* minimise |C0 + z d0 - C1 - l d1|^2 over (z, l) */
    const double w[3] = {C0[0] - C1[0], C0[1] - C1[1], C0[2] - C1[2]};
    const double a = dot3(d0, d0), b = dot3(d0, d1), c = dot3(d1, d1), d = dot3(d0, w), e = dot3(d1, w);
    const double den = a * c - b * b;
    if (!(den > 1e-12 * a * c)) return 0.0;
    return (b * e - c * d) / den;
}

static void tri_ray(const orc_tri_cam* cam, double x, double y, double C[3], double dir[3])
{
    /* C = -R^T t; dir = R^T K^-1 [x, y, 1] */
    const double k[3] = {(x - cam->cx) / cam->fx, (y - cam->cy) / cam->fy, 1.0};
    for (int r = 0; r < 3; ++r) {
        C[r] = -(cam->R[0 * 3 + r] * cam->t[0] + cam->R[1 * 3 + r] * cam->t[1] + cam->R[2 * 3 + r] * cam->t[2]);
        dir[r] = cam->R[0 * 3 + r] * k[0] + cam->R[1 * 3 + r] * k[1] + cam->R[2 * 3 + r] * k[2];
    }
}

/* angle of match s at depth z and its derivative in z */
static double tri_angle_at(const double C0[3], const double d0[3], double z, const double Cs[3], const double ds[3],
                           double* dtheta)
{
    const double a[3] = {C0[0] + z * d0[0] - Cs[0], C0[1] + z * d0[1] - Cs[1], C0[2] + z * d0[2] - Cs[2]};
    double u[3], g[3];
    cross3(a, ds, u);
    cross3(d0, ds, g);
    const double sn = sqrt(dot3(u, u)), cs = dot3(a, ds);
    const double th = atan2(sn, cs);
    if (dtheta) {
        /* theta = atan2(s, c): theta' = (c s' - s c') / (s^2 + c^2), c' = d0.ds, s' = u.(d0 x ds) / s */
        const double cp = dot3(d0, ds);
        const double sp = sn > 0.0 ? dot3(u, g) / sn : sqrt(dot3(g, g));
        *dtheta = (cs * sp - sn * cp) / (sn * sn + cs * cs);
    }
    return th;
}

int64_t orc_triangulate_pixel(const orc_tri_cam* ref, int64_t width, int64_t px, int64_t py,
                              const orc_tri_cam* src, int64_t n_src, const double* u, const double* v,
                              const double* conf, const orc_tri_opts* o, double* depth)
{
    (void)width;
    double C0[3], d0[3];
    tri_ray(ref, (double)px + 0.5, (double)py + 0.5, C0, d0);
    const double thr = o->angle_deg * M_PI / 180.0;
    double Cs[64][3], ds[64][3];
    int used[64];
    const int64_t ns = n_src < 64 ? n_src : 64;
    for (int64_t s = 0; s < ns; ++s) {
        used[s] = conf[s] >= o->conf_min;
        tri_ray(&src[s], u[s], v[s], Cs[s], ds[s]);
    }
    int64_t best_n = 0, best_s = -1;
    double best_z = 0.0;
    for (int64_t s = 0; s < ns; ++s) {
        if (!used[s]) continue;
        const double z = orc_closest_depth(C0, d0, Cs[s], ds[s]);
        if (!(z > 0.0)) continue;
        int64_t n = 0;
        for (int64_t k = 0; k < ns; ++k)
            if (used[k] && tri_angle_at(C0, d0, z, Cs[k], ds[k], NULL) < thr) ++n;
        if (n > best_n) {
            best_n = n;
            best_s = s;
            best_z = z;
        }
    }
    *depth = 0.0;
    if (best_s < 0) return 0;
    /* the inlier set of the winning hypothesis */
    int inl[64];
    for (int64_t k = 0; k < ns; ++k) inl[k] = used[k] && tri_angle_at(C0, d0, best_z, Cs[k], ds[k], NULL) < thr;
    /* minimise E(z) = sum conf * theta^2 over the inlier set: Gauss-Newton
     * direction, step halved until E decreases (near a ray's closest approach
     * the Gauss-Newton model underestimates the curvature and overshoots) */
    double z = best_z;
    double e = 0.0;
    for (int64_t k = 0; k < ns; ++k)
        if (inl[k]) {
            const double th = tri_angle_at(C0, d0, z, Cs[k], ds[k], NULL);
            e += conf[k] * th * th;
        }
    for (int64_t it = 0; it < o->refine_iters; ++it) {
        double g = 0.0, h = 0.0;
        for (int64_t k = 0; k < ns; ++k) {
            if (!inl[k]) continue;
            double dth;
            const double th = tri_angle_at(C0, d0, z, Cs[k], ds[k], &dth);
            g += conf[k] * th * dth;
            h += conf[k] * dth * dth;
        }
        if (!(h > 0.0)) break;
        double step = -g / h;
        int accepted = 0;
        for (int half = 0; half < 30; ++half, step *= 0.5) {
            const double zn = z + step;
            if (!(zn > 0.0) || !isfinite(zn)) continue;
            double en = 0.0;
            for (int64_t k = 0; k < ns; ++k)
                if (inl[k]) {
                    const double th = tri_angle_at(C0, d0, zn, Cs[k], ds[k], NULL);
                    en += conf[k] * th * th;
                }
            if (en < e) {
                z = zn;
                e = en;
                accepted = 1;
                break;
            }
        }
        if (!accepted || fabs(step) <= 1e-14 * z) break;
    }
    if (best_n > o->keep_more_than) *depth = z;
    return best_n;
}

void orc_triangulate_depth(const orc_tri_cam* ref, int64_t width, int64_t height, const orc_tri_cam* src,
                           int64_t n_src, const float* u, const float* v, const float* conf, int64_t stride,
                           const orc_tri_opts* o, double* out_depth, int64_t* out_inliers)
{
    double uu[64], vv[64], cc[64];
    const int64_t ns = n_src < 64 ? n_src : 64;
    for (int64_t py = 0; py < height; ++py)
        for (int64_t px = 0; px < width; ++px) {
            const int64_t p = py * width + px;
            for (int64_t s = 0; s < ns; ++s) {
                uu[s] = u[s * stride + p];
                vv[s] = v[s * stride + p];
                cc[s] = conf[s * stride + p];
            }
            double d;
            out_inliers[p] = orc_triangulate_pixel(ref, width, px, py, src, ns, uu, vv, cc, o, &d);
            out_depth[p] = d;
        }
}

/* ==========================================================================
 * Retrieval nearest-neighbour search -- Sec. 3.1 (precomputed global
 * retrieval features per database image) and Sec. 4.4 "Runtime" (the
 * nearest-neighbour search of retrieval features on the GPU).  FP64 dot
 * products of the bfloat16 values (each product is exact in FP64), then a
 * plain selection of the K best.
 * ========================================================================== */
double orc_bf16_to_double(uint16_t bits)
{
    /* bfloat16 = the upper 16 bits of an IEEE binary32 */
    const uint32_t u = (uint32_t)bits << 16;
    float f;
    memcpy(&f, &u, sizeof(f));
    return (double)f;
}

void orc_retrieve_topk(const uint16_t* queries, int64_t Q, const uint16_t* db, int64_t N, int64_t D,
                       int64_t K, double* out_score, int64_t* out_index)
{
    double* sc = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* qd = (double*)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
    for (int64_t q = 0; q < Q; ++q) {
        for (int64_t d = 0; d < D; ++d) qd[d] = orc_bf16_to_double(queries[q * D + d]);
        for (int64_t n = 0; n < N; ++n) {
            double s = 0.0;
            for (int64_t d = 0; d < D; ++d) s += qd[d] * orc_bf16_to_double(db[n * D + d]);
            sc[n] = s;
        }
        /* K passes of "best remaining": highest score, lowest index among equals */
        for (int64_t k = 0; k < K; ++k) {
            int64_t best = -1;
            for (int64_t n = 0; n < N; ++n) {
                if (sc[n] != sc[n]) continue; /* taken (NaN marker) */
                if (best < 0 || sc[n] > sc[best]) best = n;
            }
            out_index[q * K + k] = best;
            out_score[q * K + k] = best >= 0 ? sc[best] : 0.0;
            if (best >= 0) sc[best] = NAN;
        }
    }
    free(sc);
    free(qd);
}

/* ==========================================================================
 * Generalized absolute pose of a camera rig (supplementary "LaMAR HoloLens
 * Results": queries taken by a multi-camera rig, a GPU generalized absolute
 * pose estimator).  The rig pose is rig_from_world, X_r = R X_w + t; camera k
 * of the rig sees X_c = R_k X_r + t_k through its own pinhole intrinsics.
 * Scoring, LO, the adaptive stop and the final refinement are those of the
 * single-camera loop with every correspondence reprojected into its camera.
 * ========================================================================== */

/* real roots of sum_k c[k] x^k for deg <= 8 (Durand-Kerner on the monic
 * polynomial, Newton polish of the real ones); returns the count */
static int poly_real_roots8(const double* c_in, int deg, double* roots)
{
    double c[9];
    for (int k = 0; k <= deg; ++k) c[k] = c_in[k];
    /* only an exactly vanishing leading coefficient lowers the degree: the
     * coefficients carry powers of a length, so a small one is not negligible */
    while (deg > 0 && c[deg] == 0.0) --deg;
    if (deg == 0) return 0;
    if (deg == 1) { roots[0] = -c[0] / c[1]; return 1; }
    /* x = sigma y with sigma = |c0 / c_deg|^(1/deg): balanced coefficients, so
     * that the iteration starts near the roots whatever their scale */
    double sigma = 1.0;
    if (c[0] != 0.0) sigma = pow(fabs(c[0] / c[deg]), 1.0 / deg);
    double complex z[8];
    double a[9];
    for (int k = 0; k <= deg; ++k) a[k] = c[k] * pow(sigma, k) / (c[deg] * pow(sigma, deg));
    double bound = 1.0;
    for (int k = 0; k < deg; ++k) bound = fmax(bound, 1.0 + fabs(a[k]));
    double complex seed = 0.4 + 0.9 * I;
    double complex p = 1.0;
    for (int k = 0; k < deg; ++k) { p *= seed; z[k] = p * (0.5 * bound); }
    for (int it = 0; it < 5000; ++it) {
        double change = 0.0;
        for (int k = 0; k < deg; ++k) {
            double complex num = 0.0;
            for (int j = deg; j >= 0; --j) num = num * z[k] + a[j];
            double complex den = 1.0;
            for (int j = 0; j < deg; ++j)
                if (j != k) den *= (z[k] - z[j]);
            if (cabs(den) == 0.0) den = 1e-300;
            double complex dz = num / den;
            z[k] -= dz;
            change = fmax(change, cabs(dz) / (1.0 + cabs(z[k])));
        }
        if (change < 1e-16) break;
    }
    int nr = 0;
    for (int k = 0; k < deg; ++k) {
        if (fabs(cimag(z[k])) > 1e-3 * (1.0 + cabs(z[k]))) continue;
        double x = creal(z[k]) * sigma;
        for (int it = 0; it < 8; ++it) {
            double d = poly_deriv_eval(c, deg, x);
            if (d == 0.0) break;
            double step = poly_eval(c, deg, x) / d;
            x -= step;
            if (fabs(step) <= 1e-17 * (1.0 + fabs(x))) break;
        }
        roots[nr++] = x;
    }
    return nr;
}

static void poly_add_to(double* acc, const double* a, int da, double s)
{
    for (int k = 0; k <= da; ++k) acc[k] += s * a[k];
}

/* residuals of the three distance equations along the rays */
static void gp3p_residual(const double o[9], const double d[9], const double D2[3], const double L[3], double f[3])
{
    static const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int e = 0; e < 3; ++e) {
        int i = pr[e][0], j = pr[e][1];
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = o[3 * i + a] + L[i] * d[3 * i + a] - o[3 * j + a] - L[j] * d[3 * j + a];
        f[e] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] - D2[e];
    }
}

/* GP3P.  The points must land on the rays o_i + lambda_i d_i (rig frame,
 * |d_i| = 1).  A rigid motion keeps the pairwise distances, so for i < j
 *   |o_i + lambda_i d_i - o_j - lambda_j d_j|^2 = |X_i - X_j|^2,
 * three quadrics in the lambdas; a real solution gives a triangle congruent to
 * the world one and hence exactly one proper rigid motion.  Written out, pair
 * (i, j) reads lambda_i^2 + lambda_j^2 - 2 c lambda_i lambda_j + 2 a lambda_i
 * - 2 b lambda_j + e = 0 with c = d_i.d_j, a = d_i.(o_i - o_j),
 * b = d_j.(o_i - o_j), e = |o_i - o_j|^2 - |X_i - X_j|^2.  With lambda_1 as
 * the parameter: pair (1,2) is a monic quadratic G in lambda_2 and pair (1,3)
 * one in lambda_3; subtracting both from pair (2,3) leaves the bilinear
 * A l2 l3 + B l2 + C l3 + E = 0, so l3 = -(B l2 + E) / (A l2 + C); putting
 * that into pair (1,3) gives a second quadratic F in lambda_2; the resultant
 * of F and G in lambda_2 is a polynomial of degree 8 in lambda_1. */
int orc_gp3p(const double o[9], const double d[9], const double X[9], double R_out[72], double t_out[24],
             double lambda_out[24])
{
    double D2[3];
    static const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    double cc[3], aa[3], bb[3], ee[3];
    for (int e = 0; e < 3; ++e) {
        int i = pr[e][0], j = pr[e][1];
        double oij[3], dx[3];
        for (int a = 0; a < 3; ++a) { oij[a] = o[3 * i + a] - o[3 * j + a]; dx[a] = X[3 * i + a] - X[3 * j + a]; }
        D2[e] = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        cc[e] = d[3 * i] * d[3 * j] + d[3 * i + 1] * d[3 * j + 1] + d[3 * i + 2] * d[3 * j + 2];
        aa[e] = d[3 * i] * oij[0] + d[3 * i + 1] * oij[1] + d[3 * i + 2] * oij[2];
        bb[e] = d[3 * j] * oij[0] + d[3 * j + 1] * oij[1] + d[3 * j + 2] * oij[2];
        ee[e] = oij[0] * oij[0] + oij[1] * oij[1] + oij[2] * oij[2] - D2[e];
    }
    /* polynomials in lambda_1, ascending coefficients */
    double p[2] = {bb[0], cc[0]}, q[3] = {ee[0], 2.0 * aa[0], 1.0};   /* G: l2^2 - 2 p l2 + q */
    double r[2] = {bb[1], cc[1]}, s[3] = {ee[1], 2.0 * aa[1], 1.0};   /* l3^2 - 2 r l3 + s */
    double A = -2.0 * cc[2];
    double B[2] = {2.0 * (p[0] + aa[2]), 2.0 * p[1]};
    double Cc[2] = {2.0 * (r[0] - bb[2]), 2.0 * r[1]};
    double E[3] = {ee[2] - q[0] - s[0], -q[1] - s[1], -q[2] - s[2]};
    /* F = f2 l2^2 + f1 l2 + f0 */
    double f2[3] = {0}, f1[4] = {0}, f0[5] = {0}, tmp[5], tmp2[5];
    poly_mul(B, 1, B, 1, tmp);        poly_add_to(f2, tmp, 2, 1.0);
    poly_mul(r, 1, B, 1, tmp);        poly_add_to(f2, tmp, 2, 2.0 * A);
    poly_add_to(f2, s, 2, A * A);
    poly_mul(B, 1, E, 2, tmp);        poly_add_to(f1, tmp, 3, 2.0);
    poly_mul(B, 1, Cc, 1, tmp2);      poly_mul(r, 1, tmp2, 2, tmp); poly_add_to(f1, tmp, 3, 2.0);
    poly_mul(r, 1, E, 2, tmp);        poly_add_to(f1, tmp, 3, 2.0 * A);
    poly_mul(s, 2, Cc, 1, tmp);       poly_add_to(f1, tmp, 3, 2.0 * A);
    poly_mul(E, 2, E, 2, tmp);        poly_add_to(f0, tmp, 4, 1.0);
    poly_mul(r, 1, E, 2, tmp2);       poly_mul(tmp2, 3, Cc, 1, tmp); poly_add_to(f0, tmp, 4, 2.0);
    poly_mul(Cc, 1, Cc, 1, tmp2);     poly_mul(s, 2, tmp2, 2, tmp); poly_add_to(f0, tmp, 4, 1.0);
    /* G = l2^2 + g1 l2 + g0 */
    double g1[2] = {-2.0 * p[0], -2.0 * p[1]}, g0[3] = {q[0], q[1], q[2]};
    /* resultant of two quadratics: (f2 g0 - f0)^2 - (f2 g1 - f1)(f1 g0 - f0 g1) */
    double t1[5] = {0}, t2[4] = {0}, t3[6] = {0}, oct[9] = {0}, w[9];
    poly_mul(f2, 2, g0, 2, tmp);      poly_add_to(t1, tmp, 4, 1.0); poly_add_to(t1, f0, 4, -1.0);
    poly_mul(f2, 2, g1, 1, tmp);      poly_add_to(t2, tmp, 3, 1.0); poly_add_to(t2, f1, 3, -1.0);
    double u6[6];
    poly_mul(f1, 3, g0, 2, u6);       poly_add_to(t3, u6, 5, 1.0);
    poly_mul(f0, 4, g1, 1, u6);       poly_add_to(t3, u6, 5, -1.0);
    poly_mul(t1, 4, t1, 4, w);        poly_add_to(oct, w, 8, 1.0);
    poly_mul(t2, 3, t3, 5, w);        poly_add_to(oct, w, 8, -1.0);

    double l1s[8];
    int nr = poly_real_roots8(oct, 8, l1s);
    double sol[8][3], sol_res[8];
    int ns = 0;
    for (int k = 0; k < nr; ++k) {
        double l1 = l1s[k];
        if (!(l1 > 0.0)) continue;
        double f2v = poly_eval(f2, 2, l1), f1v = poly_eval(f1, 3, l1), f0v = poly_eval(f0, 4, l1);
        double g1v = poly_eval(g1, 1, l1), g0v = poly_eval(g0, 2, l1);
        /* lambda_2 candidates: the common root of F and G, and both roots of G
         * (the common-root formula loses accuracy when two roots are close);
         * every candidate is verified on the distance equations below */
        double l2c[3];
        int n2 = 0;
        double den = f1v - f2v * g1v;
        if (fabs(den) > 1e-12 * (fabs(f1v) + fabs(f2v * g1v) + 1e-300)) l2c[n2++] = -(f0v - f2v * g0v) / den;
        {
            /* a slightly negative discriminant from rounding: the double root */
            double disc = 0.25 * g1v * g1v - g0v;
            if (disc >= -1e-8 * (0.25 * g1v * g1v + fabs(g0v))) {
                disc = fmax(disc, 0.0);
                l2c[n2++] = -0.5 * g1v + sqrt(disc);
                l2c[n2++] = -0.5 * g1v - sqrt(disc);
            }
        }
        for (int a2 = 0; a2 < n2; ++a2) {
            double l2 = l2c[a2];
            double Bv = poly_eval(B, 1, l1), Cv = poly_eval(Cc, 1, l1), Ev = poly_eval(E, 2, l1);
            double rv = poly_eval(r, 1, l1), sv = poly_eval(s, 2, l1);
            double l3c[3];
            int n3 = 0;
            double den3 = A * l2 + Cv;
            if (fabs(den3) > 1e-12 * (fabs(A * l2) + fabs(Cv) + 1e-300)) l3c[n3++] = -(Bv * l2 + Ev) / den3;
            {
                double disc = rv * rv - sv;
                if (disc >= -1e-8 * (rv * rv + fabs(sv))) {
                    disc = fmax(disc, 0.0);
                    l3c[n3++] = rv + sqrt(disc);
                    l3c[n3++] = rv - sqrt(disc);
                }
            }
            for (int a3 = 0; a3 < n3; ++a3) {
                double L[3] = {l1, l2, l3c[a3]};
                /* Newton on the three distance equations */
                for (int it = 0; it < 50; ++it) {
                    double f[3], J[3][3] = {{0}}, dl[3];
                    gp3p_residual(o, d, D2, L, f);
                    for (int e = 0; e < 3; ++e) {
                        int i = pr[e][0], j = pr[e][1];
                        double v[3];
                        for (int a = 0; a < 3; ++a)
                            v[a] = o[3 * i + a] + L[i] * d[3 * i + a] - o[3 * j + a] - L[j] * d[3 * j + a];
                        J[e][i] = 2.0 * (v[0] * d[3 * i] + v[1] * d[3 * i + 1] + v[2] * d[3 * i + 2]);
                        J[e][j] = -2.0 * (v[0] * d[3 * j] + v[1] * d[3 * j + 1] + v[2] * d[3 * j + 2]);
                    }
                    if (!solve3(J, f, dl)) break;
                    double mx = 0.0;
                    for (int a = 0; a < 3; ++a) { L[a] -= dl[a]; mx = fmax(mx, fabs(dl[a]) / (1.0 + fabs(L[a]))); }
                    if (mx < 1e-16) break;
                }
                double f[3];
                gp3p_residual(o, d, D2, L, f);
                int ok = L[0] > 0.0 && L[1] > 0.0 && L[2] > 0.0;
                double res = 0.0;
                for (int e = 0; e < 3; ++e) {
                    ok = ok && fabs(f[e]) <= 1e-8 * (1.0 + D2[e]);
                    res = fmax(res, fabs(f[e]) / (1.0 + D2[e]));
                }
                /* one solution: closer than 1e-6 (relative) in all three depths
                 * (a nearly double solution pins down only to ~sqrt(eps)); of
                 * two such, the one with the smaller residual stays */
                for (int j = 0; j < ns && ok; ++j)
                    if (fabs(sol[j][0] - L[0]) <= 1e-6 * (1.0 + L[0]) && fabs(sol[j][1] - L[1]) <= 1e-6 * (1.0 + L[1]) &&
                        fabs(sol[j][2] - L[2]) <= 1e-6 * (1.0 + L[2])) {
                        if (res < sol_res[j]) { memcpy(sol[j], L, sizeof(L)); sol_res[j] = res; }
                        ok = 0;
                    }
                if (ok && ns < 8) { memcpy(sol[ns], L, sizeof(L)); sol_res[ns] = res; ++ns; }
            }
        }
    }
    /* ascending lambda_1 */
    for (int a = 1; a < ns; ++a)
        for (int b = a; b > 0 && sol[b][0] < sol[b - 1][0]; --b) {
            double t3s[3];
            memcpy(t3s, sol[b], sizeof(t3s));
            memcpy(sol[b], sol[b - 1], sizeof(t3s));
            memcpy(sol[b - 1], t3s, sizeof(t3s));
        }
    for (int k = 0; k < ns; ++k) {
        double P[9];
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 3; ++a) P[3 * i + a] = o[3 * i + a] + sol[k][i] * d[3 * i + a];
        horn_absolute_orientation(X, P, &R_out[9 * k], &t_out[3 * k]);
        if (lambda_out)
            for (int i = 0; i < 3; ++i) lambda_out[3 * k + i] = sol[k][i];
    }
    return ns;
}

/* X_r = R X_w + t, X_c = R_k X_r + t_k; 0 if the point is not in front of its camera */
static int rig_residual(const orc_corr* c, const int32_t* cam_of, int64_t i, const orc_rig* rig, const double R[9],
                        const double t[3], double Xr[3], double Xc[3], double r[2])
{
    const double* Xw = &c->X[3 * i];
    const int k = cam_of[i];
    const double* Rk = rig->R[k];
    const double* tk = rig->t[k];
    for (int a = 0; a < 3; ++a) Xr[a] = R[3 * a] * Xw[0] + R[3 * a + 1] * Xw[1] + R[3 * a + 2] * Xw[2] + t[a];
    for (int a = 0; a < 3; ++a) Xc[a] = Rk[3 * a] * Xr[0] + Rk[3 * a + 1] * Xr[1] + Rk[3 * a + 2] * Xr[2] + tk[a];
    if (!(Xc[2] > 0.0)) return 0;
    const orc_cam* cam = &rig->cam[k];
    r[0] = cam->fx * Xc[0] / Xc[2] + cam->cx - c->x[i];
    r[1] = cam->fy * Xc[1] / Xc[2] + cam->cy - c->y[i];
    return 1;
}

double orc_rig_score(const orc_corr* c, const int32_t* cam_of, const int64_t* idx, int64_t m, const orc_rig* rig,
                     const double R[9], const double t[3], double tau, int64_t* inliers)
{
    double tau2 = tau * tau, s = 0.0;
    int64_t cnt = 0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double Xr[3], Xc[3], r[2];
        double r2 = tau2;
        if (rig_residual(c, cam_of, i, rig, R, t, Xr, Xc, r)) {
            r2 = r[0] * r[0] + r[1] * r[1];
            if (r2 < tau2) ++cnt;
        }
        s += c->w[i] * (r2 < tau2 ? r2 : tau2);
    }
    if (inliers) *inliers = cnt;
    return s;
}

/* pixel Jacobian w.r.t. the left perturbation of the rig pose,
 * X_r' = Exp(w) X_r + v:  d X_c / d(w, v) = R_k [ -[X_r]_x | I ] */
static void rig_jacobian(const double Xr[3], const double Xc[3], const double Rk[9], const orc_cam* cam,
                         double J[2][6])
{
    double X = Xc[0], Y = Xc[1], Z = Xc[2];
    double du[3] = {cam->fx / Z, 0.0, -cam->fx * X / (Z * Z)};
    double dv[3] = {0.0, cam->fy / Z, -cam->fy * Y / (Z * Z)};
    double M[3][3] = {{0.0, Xr[2], -Xr[1]}, {-Xr[2], 0.0, Xr[0]}, {Xr[1], -Xr[0], 0.0}};
    double RM[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) RM[a][b] = Rk[3 * a] * M[0][b] + Rk[3 * a + 1] * M[1][b] + Rk[3 * a + 2] * M[2][b];
    for (int b = 0; b < 3; ++b) {
        J[0][b] = du[0] * RM[0][b] + du[1] * RM[1][b] + du[2] * RM[2][b];
        J[1][b] = dv[0] * RM[0][b] + dv[1] * RM[1][b] + dv[2] * RM[2][b];
        J[0][3 + b] = du[0] * Rk[b] + du[1] * Rk[3 + b] + du[2] * Rk[6 + b];
        J[1][3 + b] = dv[0] * Rk[b] + dv[1] * Rk[3 + b] + dv[2] * Rk[6 + b];
    }
}

static double rig_robust_cost(const orc_corr* c, const int32_t* cam_of, const int64_t* idx, int64_t m,
                              const orc_rig* rig, int loss, double tau, double cs, const double R[9],
                              const double t[3])
{
    double tau2 = tau * tau, cs2 = cs * cs, s = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double Xr[3], Xc[3], r[2], r2 = tau2;
        if (rig_residual(c, cam_of, i, rig, R, t, Xr, Xc, r)) r2 = r[0] * r[0] + r[1] * r[1];
        if (loss == LOSS_TRUNCATED) s += c->w[i] * (r2 < tau2 ? r2 : tau2);
        else s += c->w[i] * cs2 * log1p(r2 / cs2);
    }
    return s;
}

/* the Gauss-Newton schedule of the single-camera loop, rig residuals */
static int rig_gauss_newton(const orc_corr* c, const int32_t* cam_of, const int64_t* idx, int64_t m,
                            const orc_rig* rig, int loss, double tau, double cs, int64_t iters, double R[9],
                            double t[3], double* cost_io)
{
    double tau2 = tau * tau, cs2 = cs * cs;
    double cost = rig_robust_cost(c, cam_of, idx, m, rig, loss, tau, cs, R, t);
    int accepted_steps = 0;
    for (int64_t it = 0; it < iters; ++it) {
        double H[36] = {0}, g[6] = {0};
        int64_t used = 0;
        for (int64_t k = 0; k < m; ++k) {
            int64_t i = idx ? idx[k] : k;
            double Xr[3], Xc[3], r[2];
            if (!rig_residual(c, cam_of, i, rig, R, t, Xr, Xc, r)) continue;
            double r2 = r[0] * r[0] + r[1] * r[1];
            double wt;
            if (loss == LOSS_TRUNCATED) {
                if (!(r2 < tau2)) continue;
                wt = c->w[i];
            } else {
                wt = c->w[i] / (1.0 + r2 / cs2);
            }
            double J[2][6];
            rig_jacobian(Xr, Xc, rig->R[cam_of[i]], &rig->cam[cam_of[i]], J);
            for (int a = 0; a < 6; ++a) {
                g[a] += wt * (J[0][a] * r[0] + J[1][a] * r[1]);
                for (int b = 0; b < 6; ++b) H[6 * a + b] += wt * (J[0][a] * J[0][b] + J[1][a] * J[1][b]);
            }
            ++used;
        }
        if (used < 3) break;
        double mu = 0.0;
        int ok = 0;
        double d[6], Rn[9], tn[3], cn = cost;
        for (int attempt = 0; attempt < 4; ++attempt) {
            double Hd[36], mg[6];
            memcpy(Hd, H, sizeof(Hd));
            for (int a = 0; a < 6; ++a) { Hd[7 * a] += mu * H[7 * a]; mg[a] = -g[a]; }
            if (cholesky_solve6(Hd, mg, d)) {
                apply_update(d, R, t, Rn, tn);
                cn = rig_robust_cost(c, cam_of, idx, m, rig, loss, tau, cs, Rn, tn);
                if (cn < cost) { ok = 1; break; }
            }
            mu = (mu == 0.0) ? 1e-3 : mu * 10.0;
        }
        if (!ok) break;
        const double decrease = cost - cn;
        memcpy(R, Rn, sizeof(Rn));
        memcpy(t, tn, sizeof(tn));
        ++accepted_steps;
        double dn = 0;
        for (int a = 0; a < 6; ++a) dn += d[a] * d[a];
        const int converged = sqrt(dn) < 1e-10 || decrease < 1e-6 * cost;
        cost = cn;
        if (converged) break;
    }
    *cost_io = cost;
    return accepted_steps;
}

double orc_rig_lo(const orc_corr* c, const int32_t* cam_of, const int64_t* idx, int64_t m, const orc_rig* rig,
                  double tau, int64_t iters, double R[9], double t[3])
{
    double cost;
    rig_gauss_newton(c, cam_of, idx, m, rig, LOSS_TRUNCATED, tau, 1.0, iters, R, t, &cost);
    return cost;
}

int orc_rig_refine(const orc_corr* c, const int32_t* cam_of, const int64_t* sel, int64_t n_sel, const orc_rig* rig,
                   double cauchy_c, double tau, int64_t iters, double R[9], double t[3])
{
    double cost;
    return rig_gauss_newton(c, cam_of, sel, n_sel, rig, LOSS_CAUCHY, tau, cauchy_c, iters, R, t, &cost);
}

/* ray of correspondence i in the rig frame: origin = centre of its camera,
 * direction = its unit bearing rotated into the rig */
static void rig_ray(const orc_corr* c, const int32_t* cam_of, int64_t i, const orc_rig* rig, double o[3],
                    double d[3])
{
    const int k = cam_of[i];
    const orc_cam* cam = &rig->cam[k];
    const double* Rk = rig->R[k];
    const double* tk = rig->t[k];
    double b[3] = {(c->x[i] - cam->cx) / cam->fx, (c->y[i] - cam->cy) / cam->fy, 1.0};
    double n = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    for (int a = 0; a < 3; ++a) b[a] /= n;
    for (int a = 0; a < 3; ++a) {
        d[a] = Rk[a] * b[0] + Rk[3 + a] * b[1] + Rk[6 + a] * b[2];
        o[a] = -(Rk[a] * tk[0] + Rk[3 + a] * tk[1] + Rk[6 + a] * tk[2]);
    }
}

/* The LO-RANSAC loop of the single-camera case with GP3P hypotheses
 * (pose id = 8 * sample + solution index) and rig residuals. */
int orc_rig_ransac(const orc_corr* c, const int32_t* cam_of, const orc_rig* rig, const orc_opts* o,
                   orc_result* res, uint8_t* inlier_mask, int64_t* round_best_id, double* round_best_score,
                   int64_t max_rounds)
{
    memset(res, 0, sizeof(*res));
    res->best_hyp = -1;
    int64_t n = c->n;
    if (n < 3) { res->status = -1; return -1; }
    int64_t m = n < o->max_score_corr ? n : o->max_score_corr;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    orc_subsample(n, m, idx);
    int64_t total = o->max_iters, batch = o->batch;

    double best_R[9], best_t[3], best_score = INFINITY;
    int have_best = 0;
    int64_t subset_inliers = 0, hyps = 0, rounds = 0, iters = 0;
    for (int64_t r = 0;; ++r) {
        int64_t s0 = r * batch, s1 = s0 + batch < total ? s0 + batch : total;
        if (s0 >= total) break;
        double rb_score = INFINITY, rb_R[9], rb_t[3];
        int64_t rb_id = -1;
        for (int64_t s = s0; s < s1; ++s) {
            int64_t tri[3];
            if (orc_sample(o->seed, o->query_id, (uint32_t)s, m, tri) < 0) continue;
            double ro[9], rd[9], X[9];
            for (int k = 0; k < 3; ++k) {
                int64_t i = idx[tri[k]];
                rig_ray(c, cam_of, i, rig, &ro[3 * k], &rd[3 * k]);
                for (int a = 0; a < 3; ++a) X[3 * k + a] = c->X[3 * i + a];
            }
            double Rs[72], ts[24];
            int ns = orc_gp3p(ro, rd, X, Rs, ts, NULL);
            for (int k = 0; k < ns; ++k) {
                double sc = orc_rig_score(c, cam_of, idx, m, rig, &Rs[9 * k], &ts[3 * k], o->tau, NULL);
                ++hyps;
                if (sc < rb_score) {
                    rb_score = sc;
                    rb_id = 8 * s + k;
                    memcpy(rb_R, &Rs[9 * k], sizeof(rb_R));
                    memcpy(rb_t, &ts[3 * k], sizeof(rb_t));
                }
            }
        }
        if (r < max_rounds) {
            if (round_best_id) round_best_id[r] = rb_id;
            if (round_best_score) round_best_score[r] = rb_score;
        }
        if (rb_id >= 0 && rb_score < best_score) {
            memcpy(best_R, rb_R, sizeof(rb_R));
            memcpy(best_t, rb_t, sizeof(rb_t));
            best_score = rb_score;
            res->best_hyp = rb_id;
            have_best = 1;
            if (o->lo_enabled) {
                double lR[9], lt[3];
                memcpy(lR, best_R, sizeof(lR));
                memcpy(lt, best_t, sizeof(lt));
                double ls = orc_rig_lo(c, cam_of, idx, m, rig, o->tau, o->lo_iters, lR, lt);
                res->lo_count++;
                if (ls < best_score) {
                    memcpy(best_R, lR, sizeof(lR));
                    memcpy(best_t, lt, sizeof(lt));
                    best_score = ls;
                }
            }
            orc_rig_score(c, cam_of, idx, m, rig, best_R, best_t, o->tau, &subset_inliers);
        }
        iters = s1;
        rounds = r + 1;
        if (iters >= total) break;
        if (o->p_miss > 0.0 && have_best &&
            (double)iters >= orc_needed_iters((double)subset_inliers / (double)m, o->p_miss))
            break;
    }
    res->iterations = iters;
    res->rounds = rounds;
    res->hypotheses = hyps;
    if (!have_best) { free(idx); res->status = -1; return -1; }
    memcpy(res->R_best, best_R, sizeof(best_R));
    memcpy(res->t_best, best_t, sizeof(best_t));
    res->score = best_score;
    res->subset_inliers = subset_inliers;

    double R[9], t[3];
    memcpy(R, best_R, sizeof(R));
    memcpy(t, best_t, sizeof(t));
    double tau2 = o->tau * o->tau;
    if (o->final_enabled) {
        int64_t* sel = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        int64_t ns = 0;
        for (int64_t i = 0; i < n; ++i) {
            double Xr[3], Xc[3], rr[2];
            if (rig_residual(c, cam_of, i, rig, R, t, Xr, Xc, rr) && rr[0] * rr[0] + rr[1] * rr[1] < tau2)
                sel[ns++] = i;
        }
        orc_rig_refine(c, cam_of, sel, ns, rig, o->cauchy_scale, o->tau, o->final_iters, R, t);
        free(sel);
    }
    memcpy(res->R, R, sizeof(R));
    memcpy(res->t, t, sizeof(t));
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        double Xr[3], Xc[3], rr[2];
        int in = rig_residual(c, cam_of, i, rig, R, t, Xr, Xc, rr) && rr[0] * rr[0] + rr[1] * rr[1] < tau2;
        if (inlier_mask) inlier_mask[i] = (uint8_t)in;
        cnt += in;
    }
    res->num_inliers = cnt;
    free(idx);
    res->status = 0;
    return 0;
}
