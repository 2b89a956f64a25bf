/*
 * cmlbm_oracle.c -- TEST INFRASTRUCTURE ONLY (see cmlbm_oracle.h).
 *
 * Plain FP64 restatement of the D3Q27 central-moment LBM with forcing of
 * De Rosis, Huang & Coreixas, "Three-dimensional central-moments-based lattice
 * Boltzmann method with external forcing" (arXiv 1905.10182).  Every function cites
 * the section / equation it follows.  Nothing here is blocked, fused or reordered
 * beyond what those equations state; speed is not a goal.
 */
#include "cmlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q ORC_Q
static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. II below Eq. eq:truncation */

/* ---------------------------------------------------------------- lattice (Sec. II) */
/* |c_ix>, |c_iy>, |c_iz> in the order printed at the start of Sec. II. */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};

void orc_velocities(int c[Q * 3]) {
    for (int i = 0; i < Q; ++i) {
        c[3 * i + 0] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
    }
}

/* w_0 = 8/27, w_{1..6} = 2/27, w_{7..18} = 1/54, w_{19..26} = 1/216 (Sec. II, below Eq. eq:truncation) */
static double weight(int i) {
    if (i == 0) return 8.0 / 27.0;
    if (i <= 6) return 2.0 / 27.0;
    if (i <= 18) return 1.0 / 54.0;
    return 1.0 / 216.0;
}

void orc_weights(double w[Q]) {
    for (int i = 0; i < Q; ++i) w[i] = weight(i);
}

/* the direction with c_j = -c_i, found by search */
int orc_opposite(int i) {
    for (int j = 0; j < Q; ++j)
        if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) return j;
    return -1;
}

/* ------------------------------------------------------- Hermite polynomials (App. A) */
/* 1D discrete Hermite polynomials of degree 0..2 (App. A): 1, c, c^2 - c_s^2 */
static double hermite1d(int n, double c) {
    if (n == 0) return 1.0;
    if (n == 1) return c;
    return c * c - CS2;
}

/* Eq. eq:HermiteTensorProduct: H_{x..x y..y z..z} = H^(nx)(c_x) H^(ny)(c_y) H^(nz)(c_z) */
double orc_hermite(int i, int nx, int ny, int nz) {
    return hermite1d(nx, CX[i]) * hermite1d(ny, CY[i]) * hermite1d(nz, CZ[i]);
}

static double factorial(int n) { return n == 2 ? 2.0 : 1.0; } /* n in {0, 1, 2} */

static double ipow(double v, int n) {
    double r = 1.0;
    for (int k = 0; k < n; ++k) r *= v;
    return r;
}

/* --------------------------------------------------------- equilibrium, Eq. eq:truncation
 * f_i^eq = w_i rho sum over the 27 tensors H_{nx ny nz} (nx, ny, nz in 0..2, at most two per
 * axis, App. A) of H_{nx ny nz}(c_i) ux^nx uy^ny uz^nz / (nx! ny! nz! c_s^(2n)), n = nx+ny+nz:
 * the coefficient rule stated right after Eq. eq:truncation.  order < 6 drops tensors with
 * n > order (order 2 = the classical second-order equilibrium). */
void orc_equilibrium(double rho, const double u[3], int order, double feq[Q]) {
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int nz = 0; nz <= 2; ++nz)
            for (int ny = 0; ny <= 2; ++ny)
                for (int nx = 0; nx <= 2; ++nx) {
                    int n = nx + ny + nz;
                    if (n > order) continue;
                    double coef = 1.0 / (factorial(nx) * factorial(ny) * factorial(nz) * ipow(CS2, n));
                    s += coef * orc_hermite(i, nx, ny, nz) * ipow(u[0], nx) * ipow(u[1], ny) * ipow(u[2], nz);
                }
        feq[i] = weight(i) * rho * s;
    }
}

/* ------------------------------------------------------------ forcing term, Eq. forcing
 * Eq. generalForcing: F_i = w_i sum_n (1/n!) [F u^(n-1)] . H^(n).  For the tensor H_{nx ny nz}
 * the cyclic bracket [F u..u] contracts to the derivative of ux^nx uy^ny uz^nz along F:
 *   Fx nx ux^(nx-1) uy^ny uz^nz + Fy ny ux^nx uy^(ny-1) uz^nz + Fz nz ux^nx uy^ny uz^(nz-1),
 * which is exactly each bracket printed in Eq. forcing (e.g. H_xxy: 2 ux uy Fx + ux^2 Fy), with
 * the same coefficients 1/(nx! ny! nz! c_s^(2n)) as the equilibrium.
 * Reading: F is a force density and the printed rho prefactor is not applied, so that
 * sum_i F_i c_i = F, consistent with R_1 = F_x (Eq. force_cms_sixth) and Eq. macroscopic. */
void orc_forcing_term(const double F[3], const double u[3], int order, double Fi[Q]) {
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int nz = 0; nz <= 2; ++nz)
            for (int ny = 0; ny <= 2; ++ny)
                for (int nx = 0; nx <= 2; ++nx) {
                    int n = nx + ny + nz;
                    if (n == 0 || n > order) continue;
                    double coef = 1.0 / (factorial(nx) * factorial(ny) * factorial(nz) * ipow(CS2, n));
                    double bracket = 0.0;
                    if (nx > 0) bracket += F[0] * nx * ipow(u[0], nx - 1) * ipow(u[1], ny) * ipow(u[2], nz);
                    if (ny > 0) bracket += F[1] * ny * ipow(u[0], nx) * ipow(u[1], ny - 1) * ipow(u[2], nz);
                    if (nz > 0) bracket += F[2] * nz * ipow(u[0], nx) * ipow(u[1], ny) * ipow(u[2], nz - 1);
                    s += coef * orc_hermite(i, nx, ny, nz) * bracket;
                }
        Fi[i] = weight(i) * s;
    }
}

/* ------------------------------------------------------------ CM basis, Eq. basis
 * Each T_j is a signed sum of monomials cbx^a cby^b cbz^c (cb = c - u, Eq. central_directions),
 * transcribed from Eq. basis.  Monomial (a, b, c) is encoded as a + 3b + 9c. */
typedef struct { int n; int sign[3]; int mono[3]; } basis_row;
#define M(a, b, c) ((a) + 3 * (b) + 9 * (c))
static const basis_row BASIS[Q] = {
    {1, {1}, {M(0, 0, 0)}},                                   /* T0  = 1                          */
    {1, {1}, {M(1, 0, 0)}},                                   /* T1  = cbx                        */
    {1, {1}, {M(0, 1, 0)}},                                   /* T2  = cby                        */
    {1, {1}, {M(0, 0, 1)}},                                   /* T3  = cbz                        */
    {1, {1}, {M(1, 1, 0)}},                                   /* T4  = cbx cby                    */
    {1, {1}, {M(1, 0, 1)}},                                   /* T5  = cbx cbz                    */
    {1, {1}, {M(0, 1, 1)}},                                   /* T6  = cby cbz                    */
    {2, {1, -1}, {M(2, 0, 0), M(0, 2, 0)}},                   /* T7  = cbx^2 - cby^2              */
    {2, {1, -1}, {M(2, 0, 0), M(0, 0, 2)}},                   /* T8  = cbx^2 - cbz^2              */
    {3, {1, 1, 1}, {M(2, 0, 0), M(0, 2, 0), M(0, 0, 2)}},     /* T9  = cbx^2 + cby^2 + cbz^2      */
    {2, {1, 1}, {M(1, 2, 0), M(1, 0, 2)}},                    /* T10 = cbx cby^2 + cbx cbz^2      */
    {2, {1, 1}, {M(2, 1, 0), M(0, 1, 2)}},                    /* T11 = cbx^2 cby + cby cbz^2      */
    {2, {1, 1}, {M(2, 0, 1), M(0, 2, 1)}},                    /* T12 = cbx^2 cbz + cby^2 cbz      */
    {2, {1, -1}, {M(1, 2, 0), M(1, 0, 2)}},                   /* T13 = cbx cby^2 - cbx cbz^2      */
    {2, {1, -1}, {M(2, 1, 0), M(0, 1, 2)}},                   /* T14 = cbx^2 cby - cby cbz^2      */
    {2, {1, -1}, {M(2, 0, 1), M(0, 2, 1)}},                   /* T15 = cbx^2 cbz - cby^2 cbz      */
    {1, {1}, {M(1, 1, 1)}},                                   /* T16 = cbx cby cbz                */
    {3, {1, 1, 1}, {M(2, 2, 0), M(2, 0, 2), M(0, 2, 2)}},     /* T17 = x2y2 + x2z2 + y2z2         */
    {3, {1, 1, -1}, {M(2, 2, 0), M(2, 0, 2), M(0, 2, 2)}},    /* T18 = x2y2 + x2z2 - y2z2         */
    {2, {1, -1}, {M(2, 2, 0), M(2, 0, 2)}},                   /* T19 = x2y2 - x2z2                */
    {1, {1}, {M(2, 1, 1)}},                                   /* T20 = cbx^2 cby cbz              */
    {1, {1}, {M(1, 2, 1)}},                                   /* T21 = cbx cby^2 cbz              */
    {1, {1}, {M(1, 1, 2)}},                                   /* T22 = cbx cby cbz^2              */
    {1, {1}, {M(1, 2, 2)}},                                   /* T23 = cbx cby^2 cbz^2            */
    {1, {1}, {M(2, 1, 2)}},                                   /* T24 = cbx^2 cby cbz^2            */
    {1, {1}, {M(2, 2, 1)}},                                   /* T25 = cbx^2 cby^2 cbz            */
    {1, {1}, {M(2, 2, 2)}},                                   /* T26 = cbx^2 cby^2 cbz^2          */
};
#undef M

static double monomial(int m, double bx, double by, double bz) {
    return ipow(bx, m % 3) * ipow(by, (m / 3) % 3) * ipow(bz, m / 9);
}

void orc_basis(const double u[3], double T[Q * Q]) {
    for (int i = 0; i < Q; ++i) {
        double bx = CX[i] - u[0], by = CY[i] - u[1], bz = CZ[i] - u[2]; /* Eq. central_directions */
        for (int j = 0; j < Q; ++j) {
            double v = 0.0;
            for (int t = 0; t < BASIS[j].n; ++t) v += BASIS[j].sign[t] * monomial(BASIS[j].mono[t], bx, by, bz);
            T[i * Q + j] = v;
        }
    }
}

void orc_central_moments(const double u[3], const double v[Q], double k[Q]) {
    double T[Q * Q];
    orc_basis(u, T);
    for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += T[i * Q + j] * v[i];
        k[j] = s;
    }
}

/* Gaussian elimination with partial pivoting: solves A x = b, A is n x n row-major (destroyed). */
static int gauss_solve(int n, double* A, double* b, double* x) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
        if (A[piv * n + col] == 0.0) return ORC_ERR_SINGULAR;
        if (piv != col) {
            for (int c = 0; c < n; ++c) {
                double t = A[col * n + c];
                A[col * n + c] = A[piv * n + c];
                A[piv * n + c] = t;
            }
            double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < n; ++r) {
            double m = A[r * n + col] / A[col * n + col];
            if (m == 0.0) continue;
            for (int c = col; c < n; ++c) A[r * n + c] -= m * A[col * n + c];
            b[r] -= m * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int c = r + 1; c < n; ++c) s -= A[r * n + c] * x[c];
        x[r] = s / A[r * n + r];
    }
    return ORC_OK;
}

/* Eq. system: f* = (T^T)^-1 k*, solved literally */
int orc_inverse_literal(const double u[3], const double k[Q], double v[Q]) {
    double T[Q * Q], A[Q * Q], b[Q];
    orc_basis(u, T);
    for (int j = 0; j < Q; ++j) {
        for (int i = 0; i < Q; ++i) A[j * Q + i] = T[i * Q + j]; /* A = T^T */
        b[j] = k[j];
    }
    return gauss_solve(Q, A, b, v);
}

/* ------------------------------------------------------------ fast CM inverse
 * The fast CM transform the paper cites after Eq. system: T^T factors into (i) a constant map
 * B from the 27 monomial central moments kappa_abc to the basis k (read off Eq. basis) and
 * (ii) the shifted-monomial transform, a tensor product of three D1Q3 transforms.  Inverting:
 * kappa = B^-1 k, then along each axis central moments -> raw moments (binomial expansion of
 * c^n = (cb + u)^n) -> the three populations c = -1, 0, +1 (sum f = M0, sum c f = M1,
 * sum c^2 f = M2). */
static double BINV[Q * Q];
static int binv_ready = 0;

static void init_binv(void) {
    if (binv_ready) return;
    double B[Q * Q], e[Q], col[Q];
    for (int j = 0; j < Q; ++j)
        for (int m = 0; m < Q; ++m) B[j * Q + m] = 0.0;
    for (int j = 0; j < Q; ++j)
        for (int t = 0; t < BASIS[j].n; ++t) B[j * Q + BASIS[j].mono[t]] += BASIS[j].sign[t];
    for (int c = 0; c < Q; ++c) {
        double A[Q * Q];
        memcpy(A, B, sizeof(A));
        for (int r = 0; r < Q; ++r) e[r] = (r == c) ? 1.0 : 0.0;
        gauss_solve(Q, A, e, col);
        for (int r = 0; r < Q; ++r) BINV[r * Q + c] = col[r];
    }
    binv_ready = 1;
}

/* D1Q3: central moments (m0, m1, m2) at shift u -> populations p[0] (c=-1), p[1] (c=0), p[2] (c=+1) */
static void d1q3_inverse(double m0, double m1, double m2, double u, double p[3]) {
    double M0 = m0;
    double M1 = m1 + u * m0;
    double M2 = m2 + 2.0 * u * m1 + u * u * m0;
    p[1] = M0 - M2;
    p[2] = 0.5 * (M1 + M2);
    p[0] = 0.5 * (M2 - M1);
}

void orc_inverse_fast(const double u[3], const double k[Q], double v[Q]) {
    init_binv();
    double kap[Q];
    for (int m = 0; m < Q; ++m) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += BINV[m * Q + j] * k[j];
        kap[m] = s;
    }
    /* A[a][b][c]: moment orders a, b, c replaced one axis at a time by velocity index (c+1) */
    double A[3][3][3], p[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) A[a][b][c] = kap[a + 3 * b + 9 * c];
    for (int a = 0; a < 3; ++a) /* z */
        for (int b = 0; b < 3; ++b) {
            d1q3_inverse(A[a][b][0], A[a][b][1], A[a][b][2], u[2], p);
            for (int c = 0; c < 3; ++c) A[a][b][c] = p[c];
        }
    for (int a = 0; a < 3; ++a) /* y */
        for (int c = 0; c < 3; ++c) {
            d1q3_inverse(A[a][0][c], A[a][1][c], A[a][2][c], u[1], p);
            for (int b = 0; b < 3; ++b) A[a][b][c] = p[b];
        }
    for (int b = 0; b < 3; ++b) /* x */
        for (int c = 0; c < 3; ++c) {
            d1q3_inverse(A[0][b][c], A[1][b][c], A[2][b][c], u[0], p);
            for (int a = 0; a < 3; ++a) A[a][b][c] = p[a];
        }
    for (int i = 0; i < Q; ++i) v[i] = A[CX[i] + 1][CY[i] + 1][CZ[i] + 1];
}

/* ------------------------------------------------------------ collision */
/* Eq. macroscopic */
static void macroscopic_node(const double f[Q], const double F[3], double* rho, double u[3]) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        jx += f[i] * CX[i];
        jy += f[i] * CY[i];
        jz += f[i] * CZ[i];
    }
    *rho = r;
    u[0] = (jx + 0.5 * F[0]) / r;
    u[1] = (jy + 0.5 * F[1]) / r;
    u[2] = (jz + 0.5 * F[2]) / r;
}

/* Eq. eq:relaxationMatrix: Lambda = diag[1,1,1,1, w,w,w,w,w, 1,...,1] */
static void paper_lambda(double omega, double L[Q]) {
    for (int j = 0; j < Q; ++j) L[j] = (j >= 4 && j <= 8) ? omega : 1.0;
}

/* The definition (Sec. II, CMs with forcing):
 *   k* = (I - L) T^T f + L T^T feq + (I - L/2) T^T F_i,   f* = (T^T)^-1 k*  (Eq. system) */
static int collide_literal(const orc_desc* d, const double f[Q], const double F[3], double fs[Q]) {
    double rho, u[3], L[Q], feq[Q], Fi[Q], k[Q], keq[Q], R[Q], ks[Q];
    macroscopic_node(f, F, &rho, u);
    if (d->lambda) memcpy(L, d->lambda, sizeof(L));
    else paper_lambda(d->omega, L);
    orc_equilibrium(rho, u, d->eq_order, feq);
    orc_forcing_term(F, u, d->force_order, Fi);
    orc_central_moments(u, f, k);
    orc_central_moments(u, feq, keq);
    orc_central_moments(u, Fi, R);
    for (int j = 0; j < Q; ++j) ks[j] = (1.0 - L[j]) * k[j] + L[j] * keq[j] + (1.0 - 0.5 * L[j]) * R[j];
    return orc_inverse_literal(u, ks, fs);
}

/* Eq. collision: f* = f + w (feq - f) + (1 - w/2) F_i, complete feq and F_i */
static void collide_bgk(const orc_desc* d, const double f[Q], const double F[3], double fs[Q]) {
    double rho, u[3], feq[Q], Fi[Q];
    double w = d->lambda ? d->lambda[0] : d->omega;
    macroscopic_node(f, F, &rho, u);
    orc_equilibrium(rho, u, 6, feq);
    orc_forcing_term(F, u, 6, Fi);
    for (int i = 0; i < Q; ++i) fs[i] = f[i] + w * (feq[i] - f[i]) + (1.0 - 0.5 * w) * Fi[i];
}

/* The five-step time iteration summarised at the end of Sec. II, steps 1-4:
 *   1. rho, u (Eq. macroscopic);  2. k4..k8 (Eq. pre_collision);
 *   3. post-collision CMs (Eq. post_collision_central_moments_forcing);
 *   4. f* = (T^T)^-1 k* (Eq. system) through the fast CM transform. */
static void collide_paper(const orc_desc* d, const double f[Q], const double F[3], double fs[Q]) {
    double rho, u[3], ks[Q];
    macroscopic_node(f, F, &rho, u);
    double k4 = 0, k5 = 0, k6 = 0, k7 = 0, k8 = 0;
    for (int i = 0; i < Q; ++i) {
        double bx = CX[i] - u[0], by = CY[i] - u[1], bz = CZ[i] - u[2];
        k4 += f[i] * bx * by;
        k5 += f[i] * bx * bz;
        k6 += f[i] * by * bz;
        k7 += f[i] * (bx * bx - by * by);
        k8 += f[i] * (bx * bx - bz * bz);
    }
    double w = d->omega;
    for (int j = 0; j < Q; ++j) ks[j] = 0.0;
    ks[0] = rho;
    ks[1] = 0.5 * F[0];
    ks[2] = 0.5 * F[1];
    ks[3] = 0.5 * F[2];
    ks[4] = (1.0 - w) * k4;
    ks[5] = (1.0 - w) * k5;
    ks[6] = (1.0 - w) * k6;
    ks[7] = (1.0 - w) * k7;
    ks[8] = (1.0 - w) * k8;
    ks[9] = 3.0 * rho * CS2;
    ks[10] = F[0] * CS2;
    ks[11] = F[1] * CS2;
    ks[12] = F[2] * CS2;
    ks[17] = rho * CS2;
    ks[18] = rho * CS2 * CS2;
    ks[23] = 0.5 * F[0] * CS2 * CS2;
    ks[24] = 0.5 * F[1] * CS2 * CS2;
    ks[25] = 0.5 * F[2] * CS2 * CS2;
    ks[26] = rho * CS2 * CS2 * CS2;
    orc_inverse_fast(u, ks, fs);
}

int orc_collide(const orc_desc* d, const double f[Q], const double F[3], double fs[Q]) {
    init_binv();
    switch (d->collision) {
    case ORC_COLL_LITERAL: return collide_literal(d, f, F, fs);
    case ORC_COLL_PAPER: collide_paper(d, f, F, fs); return ORC_OK;
    case ORC_COLL_BGK: collide_bgk(d, f, F, fs); return ORC_OK;
    case ORC_COLL_NONE: memcpy(fs, f, sizeof(double) * Q); return ORC_OK;
    default: return ORC_ERR_ARG;
    }
}

/* ------------------------------------------------------------ grid */
typedef struct { long long N; } gridinfo;

static long long node_index(const orc_desc* d, int x, int y, int z) {
    return (long long)x + (long long)d->nx * ((long long)y + (long long)d->ny * z);
}

static int is_solid(const orc_desc* d, long long n) { return d->mask && d->mask[n]; }

/* Neighbour x + s*c_i with periodic wrap (x, z, and y without walls).
 * Returns -1 when the link leaves through a y wall or ends on a solid node. */
static long long neighbour(const orc_desc* d, int x, int y, int z, int i, int s) {
    int xn = x + s * CX[i], yn = y + s * CY[i], zn = z + s * CZ[i];
    xn = (xn % d->nx + d->nx) % d->nx;
    zn = (zn % d->nz + d->nz) % d->nz;
    if (d->walls_y) {
        if (yn < 0 || yn >= d->ny) return -1;
    } else {
        yn = (yn % d->ny + d->ny) % d->ny;
    }
    long long m = node_index(d, xn, yn, zn);
    if (is_solid(d, m)) return -1;
    return m;
}

static void gather_node(const double* f, long long N, long long n, double out[Q]) {
    for (int i = 0; i < Q; ++i) out[i] = f[(long long)i * N + n];
}

/* psi = 1 - exp(-rho) of the static-droplet test (Sec. III) */
static void compute_psi(const orc_desc* d, const double* f, double* psi) {
    long long N = (long long)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double r = 0.0;
        for (int i = 0; i < Q; ++i) r += f[(long long)i * N + n];
        psi[n] = 1.0 - exp(-r);
    }
}

/* Force density at node n. */
static void node_force(const orc_desc* d, const double* psi, int x, int y, int z, double F[3]) {
    long long n = node_index(d, x, y, z);
    F[0] = F[1] = F[2] = 0.0;
    switch (d->force_kind) {
    case ORC_FORCE_UNIFORM:
        F[0] = d->force[0];
        F[1] = d->force[1];
        F[2] = d->force[2];
        break;
    case ORC_FORCE_KOLMOGOROV:
        F[0] = d->force[0] * sin(2.0 * M_PI * (double)y / (double)d->ny);
        break;
    case ORC_FORCE_FIELD:
        F[0] = d->fx[n];
        F[1] = d->fy[n];
        F[2] = d->fz[n];
        break;
    case ORC_FORCE_SHAN_CHEN: {
        /* F = -G psi(x) sum_i w_i c_i psi(x + c_i), periodic (Sec. III, static droplet) */
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int i = 0; i < Q; ++i) {
            long long m = neighbour(d, x, y, z, i, +1);
            double w = weight(i);
            sx += w * CX[i] * psi[m];
            sy += w * CY[i] * psi[m];
            sz += w * CZ[i] * psi[m];
        }
        F[0] = -d->G * psi[n] * sx;
        F[1] = -d->G * psi[n] * sy;
        F[2] = -d->G * psi[n] * sz;
        break;
    }
    default: break;
    }
}

static int check_desc(const orc_desc* d) {
    if (!d || d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return ORC_ERR_ARG;
    if (d->force_kind == ORC_FORCE_SHAN_CHEN && (d->walls_y || d->mask)) return ORC_ERR_ARG;
    if (d->force_kind == ORC_FORCE_FIELD && (!d->fx || !d->fy || !d->fz)) return ORC_ERR_ARG;
    if (d->collision < 0 || d->collision > ORC_COLL_NONE) return ORC_ERR_ARG;
    if (d->threads > 0) {
#ifdef _OPENMP
        omp_set_num_threads(d->threads);
#endif
    }
    init_binv();
    return ORC_OK;
}

int orc_force_field(const orc_desc* d, const double* f, double* F3) {
    int st = check_desc(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
    double* psi = NULL;
    if (d->force_kind == ORC_FORCE_SHAN_CHEN) {
        psi = (double*)malloc(sizeof(double) * N);
        if (!psi) return ORC_ERR_NOMEM;
        compute_psi(d, f, psi);
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < d->nz; ++z)
        for (int y = 0; y < d->ny; ++y)
            for (int x = 0; x < d->nx; ++x) {
                long long n = node_index(d, x, y, z);
                double F[3];
                node_force(d, psi, x, y, z, F);
                F3[n] = F[0];
                F3[N + n] = F[1];
                F3[2 * N + n] = F[2];
            }
    free(psi);
    return ORC_OK;
}

int orc_macroscopic(const orc_desc* d, const double* f, double* rho, double* u3) {
    long long N = (long long)d->nx * d->ny * d->nz;
    double* F3 = (double*)malloc(sizeof(double) * 3 * N);
    if (!F3) return ORC_ERR_NOMEM;
    int st = orc_force_field(d, f, F3);
    if (st) {
        free(F3);
        return st;
    }
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double fl[Q], F[3] = {F3[n], F3[N + n], F3[2 * N + n]}, r, u[3];
        gather_node(f, N, n, fl);
        macroscopic_node(fl, F, &r, u);
        rho[n] = r;
        u3[n] = u[0];
        u3[N + n] = u[1];
        u3[2 * N + n] = u[2];
    }
    free(F3);
    return ORC_OK;
}

int orc_init_equilibrium(const orc_desc* d, const double* rho, const double* u3, double* f) {
    int st = check_desc(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double feq[Q], u[3] = {u3[n], u3[N + n], u3[2 * N + n]}, r = rho[n];
        if (is_solid(d, n)) {
            u[0] = u[1] = u[2] = 0.0;
            r = d->rho0;
        }
        orc_equilibrium(r, u, 6, feq);
        for (int i = 0; i < Q; ++i) f[(long long)i * N + n] = feq[i];
    }
    return ORC_OK;
}

/* Eq. streaming, f_i(x + c_i, t+1) = f*_i(x, t), written as a pull from x - c_i; a link whose
 * source lies behind a wall or on a solid node takes the bounced-back population f*_opp(i)(x, t)
 * (halfway bounce-back). */
int orc_step(const orc_desc* d, double* f, int nsteps) {
    int st = check_desc(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
    double* fs = (double*)malloc(sizeof(double) * Q * N);
    double* psi = (d->force_kind == ORC_FORCE_SHAN_CHEN) ? (double*)malloc(sizeof(double) * N) : NULL;
    if (!fs || (d->force_kind == ORC_FORCE_SHAN_CHEN && !psi)) {
        free(fs);
        free(psi);
        return ORC_ERR_NOMEM;
    }
    int err = ORC_OK;
    for (int s = 0; s < nsteps && !err; ++s) {
        if (psi) compute_psi(d, f, psi);
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int z = 0; z < d->nz; ++z)
            for (int y = 0; y < d->ny; ++y)
                for (int x = 0; x < d->nx; ++x) {
                    long long n = node_index(d, x, y, z);
                    double fl[Q], fo[Q], F[3];
                    gather_node(f, N, n, fl);
                    if (is_solid(d, n)) {
                        for (int i = 0; i < Q; ++i) fs[(long long)i * N + n] = fl[i];
                        continue;
                    }
                    node_force(d, psi, x, y, z, F);
                    err |= orc_collide(d, fl, F, fo);
                    for (int i = 0; i < Q; ++i) fs[(long long)i * N + n] = fo[i];
                }
#pragma omp parallel for schedule(static)
        for (int z = 0; z < d->nz; ++z)
            for (int y = 0; y < d->ny; ++y)
                for (int x = 0; x < d->nx; ++x) {
                    long long n = node_index(d, x, y, z);
                    if (is_solid(d, n)) continue;
                    for (int i = 0; i < Q; ++i) {
                        long long src = neighbour(d, x, y, z, i, -1);
                        f[(long long)i * N + n] = (src >= 0) ? fs[(long long)i * N + src]
                                                             : fs[(long long)orc_opposite(i) * N + n];
                    }
                }
    }
    free(fs);
    free(psi);
    return err;
}

int orc_step_sampled(const orc_desc* d, const double* f, const long long* nodes, int count, double* out) {
    int st = check_desc(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
    double* psi = NULL;
    if (d->force_kind == ORC_FORCE_SHAN_CHEN) {
        psi = (double*)malloc(sizeof(double) * N);
        if (!psi) return ORC_ERR_NOMEM;
        compute_psi(d, f, psi);
    }
    int err = ORC_OK;
#pragma omp parallel for schedule(dynamic) reduction(| : err)
    for (int k = 0; k < count; ++k) {
        long long n = nodes[k];
        int x = (int)(n % d->nx), y = (int)((n / d->nx) % d->ny), z = (int)(n / ((long long)d->nx * d->ny));
        double fl[Q], fo[Q], F[3];
        if (is_solid(d, n)) {
            gather_node(f, N, n, fl);
            for (int i = 0; i < Q; ++i) out[(long long)k * Q + i] = fl[i];
            continue;
        }
        for (int i = 0; i < Q; ++i) {
            long long src = neighbour(d, x, y, z, i, -1);
            int dir = i;
            long long at = src;
            int sx = x - CX[i], sy = y - CY[i], sz = z - CZ[i];
            if (src < 0) { /* bounce-back: f*_opp(i) of this node */
                dir = orc_opposite(i);
                at = n;
                sx = x;
                sy = y;
                sz = z;
            }
            sx = (sx % d->nx + d->nx) % d->nx;
            sy = (sy % d->ny + d->ny) % d->ny;
            sz = (sz % d->nz + d->nz) % d->nz;
            gather_node(f, N, at, fl);
            node_force(d, psi, sx, sy, sz, F);
            err |= orc_collide(d, fl, F, fo);
            out[(long long)k * Q + i] = fo[dir];
        }
    }
    free(psi);
    return err;
}

/* ------------------------------------------------------------------ magnetic field (App. C) */
static const int XI[ORC_QM][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double CSM2 = 0.25; /* c_s^2 of D3Q7 (c_s = 1/2, App. C) */

static double wm(int l) { return l == 0 ? 0.25 : 0.125; }
static int opp_m(int l) { return l == 0 ? 0 : (l % 2 ? l + 1 : l - 1); }

void orc_mhd_velocities(int xi[ORC_QM * 3]) {
    for (int l = 0; l < ORC_QM; ++l)
        for (int a = 0; a < 3; ++a) xi[3 * l + a] = XI[l][a];
}

void orc_mhd_weights(double w[ORC_QM]) {
    for (int l = 0; l < ORC_QM; ++l) w[l] = wm(l);
}

/* App. C: h_la^eq = w_l [b_a + 4 xi_lb (u_b b_a - b_b u_a)] */
void orc_mhd_equilibrium(const double b[3], const double u[3], double heq[ORC_QM * 3]) {
    for (int l = 0; l < ORC_QM; ++l)
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += XI[l][c] * (u[c] * b[a] - b[c] * u[a]);
            heq[3 * l + a] = wm(l) * (b[a] + 4.0 * s);
        }
}

void orc_mhd_moments(const double h[ORC_QM * 3], double b[3], double E[3]) {
    double L[3][3] = {{0}}; /* electric tensor L[beta][alpha] = sum_l xi_lb h_la */
    b[0] = b[1] = b[2] = 0.0;
    for (int l = 0; l < ORC_QM; ++l)
        for (int a = 0; a < 3; ++a) {
            b[a] += h[3 * l + a];
            for (int c = 0; c < 3; ++c) L[c][a] += XI[l][c] * h[3 * l + a];
        }
    /* E_g = eps_gba L[b][a] */
    E[0] = L[1][2] - L[2][1];
    E[1] = L[2][0] - L[0][2];
    E[2] = L[0][1] - L[1][0];
}

static void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_mhd_node(const double f[ORC_Q], const double h[ORC_QM * 3], const double Fext[3], double omega_m,
                  double* rho, double u[3], double FL[3], double j[3]) {
    double r = 0.0, m1[3] = {0, 0, 0}, b[3], E[3], Exb[3], s[3];
    for (int i = 0; i < ORC_Q; ++i) {
        r += f[i];
        m1[0] += f[i] * CX[i];
        m1[1] += f[i] * CY[i];
        m1[2] += f[i] * CZ[i];
    }
    orc_mhd_moments(h, b, E);
    const double kappa = omega_m / CSM2;
    cross(E, b, Exb);
    /* rho u = m1 + F_ext/2 + F_L/2 with F_L = -kappa E x b + 2 kappa ((u.b) b - |b|^2 u):
       the component of u along b sees rho, the perpendicular part rho + kappa |b|^2 */
    for (int a = 0; a < 3; ++a) s[a] = m1[a] + 0.5 * Fext[a] - 0.5 * kappa * Exb[a];
    const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    if (bb > 0.0) {
        const double sb = (s[0] * b[0] + s[1] * b[1] + s[2] * b[2]) / bb;
        for (int a = 0; a < 3; ++a) {
            const double par = sb * b[a];
            u[a] = par / r + (s[a] - par) / (r + kappa * bb);
        }
    } else {
        for (int a = 0; a < 3; ++a) u[a] = s[a] / r;
    }
    double uxb[3];
    cross(u, b, uxb);
    for (int a = 0; a < 3; ++a) j[a] = -kappa * (E[a] - 2.0 * uxb[a]);
    cross(j, b, FL);
    *rho = r;
}

static int check_mhd(const orc_desc* d) {
    int st = check_desc(d);
    if (st) return st;
    if (d->mask || (d->force_kind != ORC_FORCE_NONE && d->force_kind != ORC_FORCE_UNIFORM)) return ORC_ERR_ARG;
    return ORC_OK;
}

static void gather_h(const double* h, long long N, long long n, double out[ORC_QM * 3]) {
    for (int k = 0; k < 3 * ORC_QM; ++k) out[k] = h[(long long)k * N + n];
}

int orc_mhd_init(const orc_desc* d, const double* b3, const double* u3, double* h) {
    int st = check_mhd(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double b[3] = {b3[n], b3[N + n], b3[2 * N + n]}, u[3] = {u3[n], u3[N + n], u3[2 * N + n]}, heq[3 * ORC_QM];
        orc_mhd_equilibrium(b, u, heq);
        for (int k = 0; k < 3 * ORC_QM; ++k) h[(long long)k * N + n] = heq[k];
    }
    return ORC_OK;
}

int orc_mhd_step(const orc_desc* d, double omega_m, const double b_wall[3], double* f, double* h, int nsteps) {
    int st = check_mhd(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
    double* fs = (double*)malloc(sizeof(double) * Q * N);
    double* hs = (double*)malloc(sizeof(double) * 3 * ORC_QM * N);
    if (!fs || !hs) {
        free(fs);
        free(hs);
        return ORC_ERR_NOMEM;
    }
    const double Fext[3] = {d->force_kind == ORC_FORCE_UNIFORM ? d->force[0] : 0.0,
                            d->force_kind == ORC_FORCE_UNIFORM ? d->force[1] : 0.0,
                            d->force_kind == ORC_FORCE_UNIFORM ? d->force[2] : 0.0};
    int err = ORC_OK;
    for (int s = 0; s < nsteps && !err; ++s) {
        /* collision of both populations */
#pragma omp parallel for schedule(static) reduction(| : err)
        for (long long n = 0; n < N; ++n) {
            double fl[Q], fo[Q], hl[3 * ORC_QM], heq[3 * ORC_QM], rho, u[3], FL[3], j[3], F[3], b[3], E[3];
            gather_node(f, N, n, fl);
            gather_h(h, N, n, hl);
            orc_mhd_node(fl, hl, Fext, omega_m, &rho, u, FL, j);
            for (int a = 0; a < 3; ++a) F[a] = Fext[a] + FL[a];
            err |= orc_collide(d, fl, F, fo);
            for (int i = 0; i < Q; ++i) fs[(long long)i * N + n] = fo[i];
            orc_mhd_moments(hl, b, E);
            orc_mhd_equilibrium(b, u, heq);
            for (int k = 0; k < 3 * ORC_QM; ++k) hs[(long long)k * N + n] = hl[k] + omega_m * (heq[k] - hl[k]);
        }
        /* streaming: pull from x - c; fluid halfway bounce-back, magnetic anti-bounce-back at walls */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < d->nz; ++z)
            for (int y = 0; y < d->ny; ++y)
                for (int x = 0; x < d->nx; ++x) {
                    long long n = node_index(d, x, y, z);
                    for (int i = 0; i < Q; ++i) {
                        long long src = neighbour(d, x, y, z, i, -1);
                        f[(long long)i * N + n] = (src >= 0) ? fs[(long long)i * N + src]
                                                             : fs[(long long)orc_opposite(i) * N + n];
                    }
                    for (int l = 0; l < ORC_QM; ++l) {
                        /* D3Q7 velocity l is D3Q27 velocity l (the first seven of Sec. II) */
                        long long src = neighbour(d, x, y, z, l, -1);
                        for (int a = 0; a < 3; ++a) {
                            h[(long long)(3 * l + a) * N + n] =
                                (src >= 0) ? hs[(long long)(3 * l + a) * N + src]
                                           : -hs[(long long)(3 * opp_m(l) + a) * N + n] + 2.0 * wm(l) * b_wall[a];
                        }
                    }
                }
    }
    free(fs);
    free(hs);
    return err;
}

int orc_mhd_fields(const orc_desc* d, double omega_m, const double* f, const double* h, double* rho, double* u3,
                   double* b3, double* j3) {
    int st = check_mhd(d);
    if (st) return st;
    long long N = (long long)d->nx * d->ny * d->nz;
    const double Fext[3] = {d->force_kind == ORC_FORCE_UNIFORM ? d->force[0] : 0.0,
                            d->force_kind == ORC_FORCE_UNIFORM ? d->force[1] : 0.0,
                            d->force_kind == ORC_FORCE_UNIFORM ? d->force[2] : 0.0};
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double fl[Q], hl[3 * ORC_QM], r, u[3], FL[3], j[3], b[3], E[3];
        gather_node(f, N, n, fl);
        gather_h(h, N, n, hl);
        orc_mhd_node(fl, hl, Fext, omega_m, &r, u, FL, j);
        orc_mhd_moments(hl, b, E);
        rho[n] = r;
        for (int a = 0; a < 3; ++a) {
            u3[a * N + n] = u[a];
            b3[a * N + n] = b[a];
            j3[a * N + n] = j[a];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ colour gradient (App. D) */
static int shell(int i) { return CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]; }

void orc_cg_phi(double alpha, double phi_i[Q]) {
    for (int i = 0; i < Q; ++i) {
        switch (shell(i)) {
        case 0: phi_i[i] = alpha; break;
        case 1: phi_i[i] = 2.0 * (1.0 - alpha) / 19.0; break;
        case 2: phi_i[i] = (1.0 - alpha) / 38.0; break;
        default: phi_i[i] = (1.0 - alpha) / 152.0; break;
        }
    }
}

void orc_cg_equilibrium(double rho, const double u[3], double alpha, double nu, const double grad_rho[3],
                        double feq[Q]) {
    double phi_i[Q], fc[Q];
    orc_cg_phi(alpha, phi_i);
    orc_equilibrium(rho, u, 6, fc);
    const double ug = u[0] * grad_rho[0] + u[1] * grad_rho[1] + u[2] * grad_rho[2];
    for (int i = 0; i < Q; ++i) {
        /* G : c c with G = (u grad rho + grad rho u) / 48 */
        const double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        const double cg = CX[i] * grad_rho[0] + CY[i] * grad_rho[1] + CZ[i] * grad_rho[2];
        const double Gcc = 2.0 * cu * cg / 48.0;
        double Phi;
        switch (shell(i)) {
        case 0: Phi = -3.0 * nu * ug; break;
        case 1: Phi = 16.0 * nu * Gcc; break;
        case 2: Phi = 4.0 * nu * Gcc; break;
        default: Phi = nu * Gcc; break;
        }
        feq[i] = rho * phi_i[i] + (fc[i] - rho * weight(i)) + Phi;
    }
}

void orc_cg_perturbation(double A, const double gp[3], double out[Q]) {
    const double g2 = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
    for (int i = 0; i < Q; ++i) out[i] = 0.0;
    if (!(g2 > 0.0)) return;
    const double gn = sqrt(g2);
    for (int i = 0; i < Q; ++i) {
        const double cg = CX[i] * gp[0] + CY[i] * gp[1] + CZ[i] * gp[2];
        double B;
        switch (shell(i)) {
        case 0: B = -10.0 / 27.0; break;
        case 1: B = 2.0 / 27.0; break;
        case 2: B = 1.0 / 54.0; break;
        default: B = 1.0 / 216.0; break;
        }
        out[i] = 0.5 * A * gn * (weight(i) * cg * cg / g2 - B);
    }
}

void orc_cg_recolour(double beta, double rho_r, double rho_b, double alpha, const double gp[3], const double fs[Q],
                     double fr[Q], double fb[Q]) {
    const double rho = rho_r + rho_b;
    double phi_i[Q];
    orc_cg_phi(alpha, phi_i);
    const double gn = sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
    for (int i = 0; i < Q; ++i) {
        double cosv = 0.0;
        if (gn > 0.0 && shell(i) > 0)
            cosv = (CX[i] * gp[0] + CY[i] * gp[1] + CZ[i] * gp[2]) / (sqrt((double)shell(i)) * gn);
        fr[i] = rho_r / rho * fs[i] + beta * rho_r * rho_b / (rho * rho) * cosv * rho * phi_i[i];
        fb[i] = fs[i] - fr[i];
    }
}

static double cg_order(const orc_cg* m, double rr, double rb) {
    const double a = rr / m->rho_r0, b = rb / m->rho_b0;
    return (a - b) / (a + b);
}

static void cg_params(const orc_cg* m, double phi, double* alpha, double* nu) {
    const double ab = 8.0 / 27.0;
    const double ar = 1.0 - (1.0 - ab) * m->rho_b0 / m->rho_r0;
    *alpha = 0.5 * (1.0 + phi) * ar + 0.5 * (1.0 - phi) * ab;
    *nu = 1.0 / (0.5 * (1.0 + phi) / m->nu_r + 0.5 * (1.0 - phi) / m->nu_b);
}

/* isotropic central gradient of a node field; a neighbour behind a wall takes the node's value */
static void cg_gradient(const orc_desc* d, const double* X, int x, int y, int z, double g[3]) {
    const long long n = node_index(d, x, y, z);
    g[0] = g[1] = g[2] = 0.0;
    for (int i = 1; i < Q; ++i) {
        long long mnb = neighbour(d, x, y, z, i, +1);
        const double v = mnb >= 0 ? X[mnb] : X[n];
        g[0] += weight(i) * CX[i] * v / CS2;
        g[1] += weight(i) * CY[i] * v / CS2;
        g[2] += weight(i) * CZ[i] * v / CS2;
    }
}

static int check_cg(const orc_cg* m) {
    if (!m || !m->grid) return ORC_ERR_ARG;
    if (!(m->rho_r0 > 0.0) || !(m->rho_b0 > 0.0) || !(m->nu_r > 0.0) || !(m->nu_b > 0.0)) return ORC_ERR_ARG;
    if (m->grid->mask) return ORC_ERR_ARG;
    return check_desc(m->grid);
}

int orc_cg_init(const orc_cg* m, const double* rho_r, const double* rho_b, const double* u3, double* fr, double* fb) {
    int st = check_cg(m);
    if (st) return st;
    const orc_desc* d = m->grid;
    long long N = (long long)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        const double rr = rho_r[n], rb = rho_b[n], rho = rr + rb;
        double alpha, nu, feq[Q], u[3] = {u3[n], u3[N + n], u3[2 * N + n]}, g0[3] = {0, 0, 0};
        cg_params(m, cg_order(m, rr, rb), &alpha, &nu);
        orc_cg_equilibrium(rho, u, alpha, nu, g0, feq);
        for (int i = 0; i < Q; ++i) {
            fr[(long long)i * N + n] = rr / rho * feq[i];
            fb[(long long)i * N + n] = rb / rho * feq[i];
        }
    }
    return ORC_OK;
}

/* per-node fields of the current state: rho_r, rho_b, rho, phi */
static void cg_node_fields(const orc_cg* m, const double* fr, const double* fb, long long N, double* rr, double* rb,
                           double* rho, double* phi) {
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < Q; ++i) {
            a += fr[(long long)i * N + n];
            b += fb[(long long)i * N + n];
        }
        rr[n] = a;
        rb[n] = b;
        rho[n] = a + b;
        phi[n] = cg_order(m, a, b);
    }
}

static void cg_force(const orc_cg* m, double rho, double F[3]) {
    const double dr = rho - 0.5 * (m->rho_r0 + m->rho_b0);
    F[0] = dr * m->gvec[0];
    F[1] = dr * m->gvec[1];
    F[2] = dr * m->gvec[2];
}

int orc_cg_step(const orc_cg* m, double* fr, double* fb, int nsteps) {
    int st = check_cg(m);
    if (st) return st;
    const orc_desc* d = m->grid;
    long long N = (long long)d->nx * d->ny * d->nz;
    double* frs = (double*)malloc(sizeof(double) * Q * N);
    double* fbs = (double*)malloc(sizeof(double) * Q * N);
    double* fld = (double*)malloc(sizeof(double) * 4 * N);
    if (!frs || !fbs || !fld) {
        free(frs);
        free(fbs);
        free(fld);
        return ORC_ERR_NOMEM;
    }
    double *rr = fld, *rb = fld + N, *rhof = fld + 2 * N, *phif = fld + 3 * N;
    int err = ORC_OK;
    for (int s = 0; s < nsteps && !err; ++s) {
        cg_node_fields(m, fr, fb, N, rr, rb, rhof, phif);
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int z = 0; z < d->nz; ++z)
            for (int y = 0; y < d->ny; ++y)
                for (int x = 0; x < d->nx; ++x) {
                    const long long n = node_index(d, x, y, z);
                    double f[Q], F[3], gphi[3], grho[3], alpha, nu, rho, u[3], feq[Q], Fi[Q], k[Q], keq[Q], R[Q],
                        ks[Q], fs[Q], pert[Q], ofr[Q], ofb[Q], L[Q];
                    for (int i = 0; i < Q; ++i) f[i] = fr[(long long)i * N + n] + fb[(long long)i * N + n];
                    cg_force(m, rhof[n], F);
                    macroscopic_node(f, F, &rho, u);
                    cg_gradient(d, phif, x, y, z, gphi);
                    cg_gradient(d, rhof, x, y, z, grho);
                    cg_params(m, phif[n], &alpha, &nu);
                    /* single phase (App. D): the CM collision of Sec. II with the enhanced equilibrium */
                    orc_cg_equilibrium(rho, u, alpha, nu, grho, feq);
                    orc_forcing_term(F, u, 6, Fi);
                    paper_lambda(1.0 / (3.0 * nu + 0.5), L);
                    orc_central_moments(u, f, k);
                    orc_central_moments(u, feq, keq);
                    orc_central_moments(u, Fi, R);
                    for (int j = 0; j < Q; ++j) ks[j] = (1.0 - L[j]) * k[j] + L[j] * keq[j] + (1.0 - 0.5 * L[j]) * R[j];
                    orc_inverse_fast(u, ks, fs); /* equals the literal solve (pinned) */
                    /* perturbation, then recolouring */
                    orc_cg_perturbation(m->A, gphi, pert);
                    for (int i = 0; i < Q; ++i) fs[i] += pert[i];
                    orc_cg_recolour(m->beta, rr[n], rb[n], alpha, gphi, fs, ofr, ofb);
                    for (int i = 0; i < Q; ++i) {
                        frs[(long long)i * N + n] = ofr[i];
                        fbs[(long long)i * N + n] = ofb[i];
                    }
                }
#pragma omp parallel for schedule(static)
        for (int z = 0; z < d->nz; ++z)
            for (int y = 0; y < d->ny; ++y)
                for (int x = 0; x < d->nx; ++x) {
                    const long long n = node_index(d, x, y, z);
                    for (int i = 0; i < Q; ++i) {
                        const long long src = neighbour(d, x, y, z, i, -1);
                        const long long a = (long long)i * N, o = (long long)orc_opposite(i) * N;
                        fr[a + n] = src >= 0 ? frs[a + src] : frs[o + n];
                        fb[a + n] = src >= 0 ? fbs[a + src] : fbs[o + n];
                    }
                }
    }
    free(frs);
    free(fbs);
    free(fld);
    return err;
}

int orc_cg_fields(const orc_cg* m, const double* fr, const double* fb, double* rho_r, double* rho_b, double* u3) {
    int st = check_cg(m);
    if (st) return st;
    const orc_desc* d = m->grid;
    long long N = (long long)d->nx * d->ny * d->nz;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < N; ++n) {
        double f[Q], F[3], rho, u[3], a = 0.0, b = 0.0;
        for (int i = 0; i < Q; ++i) {
            a += fr[(long long)i * N + n];
            b += fb[(long long)i * N + n];
            f[i] = fr[(long long)i * N + n] + fb[(long long)i * N + n];
        }
        cg_force(m, a + b, F);
        macroscopic_node(f, F, &rho, u);
        rho_r[n] = a;
        rho_b[n] = b;
        u3[n] = u[0];
        u3[N + n] = u[1];
        u3[2 * N + n] = u[2];
    }
    return ORC_OK;
}
