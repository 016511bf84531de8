/*
 * wtmd_oracle.c -- plain, slow, FP64 CPU oracle for the well-tempered
 * metadynamics (WTMD) bias-force path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header,
 * constant or table with the CUDA library; the two are written independently
 * and compared on the same seeded inputs.
 *
 * Every function follows the plain definition of what it computes, in the
 * order the definition states it, in double precision:
 *   - metadynamics bias as a sum of Gaussians deposited at intervals, fixed
 *     height (standard) or height scaled by a bias factor (well-tempered):
 *     PySAGES paper, Sec. 2.1.5 "Metadynamics";
 *   - optional storage of the bias on a pre-defined grid: Sec. 2.1.5;
 *   - free energy A(xi) = -kT ln p(xi) + C: Sec. 2.1, Eq. (free-energy);
 *   - collective variables (Component, DihedralAngle, RadiusofGyration):
 *     Sec. 2.2; their gradients (the paper obtains them with jax.grad,
 *     Sec. 2) are written here analytically and pinned by finite differences;
 *   - the bias force is added to the engine's net force each step: Sec. 2
 *     ("force-like object ... biasing forces are added to the backend net
 *     forces"); the step structure (half-step integration, bonded and pair
 *     forces, CV, bias-force addition, second half-step) is the one named in
 *     Sec. 3.2.1.
 * Readings where the paper is silent (WT height formula, coordination
 * switching function, Philox counter layout, BAOAB splitting, deposition
 * timing) are stated at each function.
 *
 * Parity pins (tests/test_oracle_*.py): Philox known-answer vectors,
 * Mueller-Brown minima, closed forms of single hills, finite-difference
 * Jacobians, translation/rotation invariances, the WT fixed-point recursion,
 * the BAOAB harmonic-oscillator variance, and recovery of the Mueller-Brown
 * free energy from -(gamma/(gamma-1)) V.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as */
/* easy as 1, 2, 3", SC'11.  Round: two 32x32->64 products of counter words */
/* 0 and 2 with the multipliers; outputs mix the high halves with the other */
/* counter words and the key; the key advances by the Weyl constants        */
/* between rounds.                                                          */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Noise stream of the Langevin thermostat (reading: the paper fixes no RNG).
 * key = (seed low word, seed high word); counter = (step low word, global
 * particle index, step high word, 0).  The four 32-bit outputs become
 * uniforms u = (x + 1/2) / 2^32 in (0,1) and two Box-Muller pairs; the first
 * three normals drive x, y, z. */
void orc_noise3(uint64_t seed, uint64_t step, uint32_t particle, double g[3])
{
    uint32_t ctr[4] = {(uint32_t)step, particle, (uint32_t)(step >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u[4];
    for (int i = 0; i < 4; ++i) u[i] = ((double)r[i] + 0.5) / 4294967296.0;
    double rad0 = sqrt(-2.0 * log(u[0]));
    double rad1 = sqrt(-2.0 * log(u[2]));
    g[0] = rad0 * cos(2.0 * ORC_PI * u[1]);
    g[1] = rad0 * sin(2.0 * ORC_PI * u[1]);
    g[2] = rad1 * cos(2.0 * ORC_PI * u[3]);
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------ */
/* d = a - b, minimum image in each periodic dimension (box[k] > 0). */
static void orc_delta(const double* a, const double* b, const double* box, double d[3])
{
    for (int k = 0; k < 3; ++k) {
        d[k] = a[k] - b[k];
        if (box && box[k] > 0.0) d[k] -= box[k] * nearbyint(d[k] / box[k]);
    }
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* Engines (the systems that drive the method; the paper's backends own     */
/* these).                                                                  */
/* ------------------------------------------------------------------------ */

/* Mueller-Brown potential (Mueller & Brown, Theor. Chim. Acta 53, 75 (1979)):
 * U(x,y) = sum_k A_k exp(a_k (x-x_k)^2 + b_k (x-x_k)(y-y_k) + c_k (y-y_k)^2). */
static const double MB_A[4] = {-200.0, -100.0, -170.0, 15.0};
static const double MB_a[4] = {-1.0, -1.0, -6.5, 0.7};
static const double MB_b[4] = {0.0, 0.0, 11.0, 0.6};
static const double MB_c[4] = {-10.0, -10.0, -6.5, 0.7};
static const double MB_x0[4] = {1.0, 0.0, -0.5, -1.0};
static const double MB_y0[4] = {0.0, 0.5, 1.5, 1.0};

double orc_mb(double x, double y, double* fx, double* fy)
{
    double U = 0.0, gx = 0.0, gy = 0.0;
    for (int k = 0; k < 4; ++k) {
        double dx = x - MB_x0[k], dy = y - MB_y0[k];
        double e = MB_A[k] * exp(MB_a[k] * dx * dx + MB_b[k] * dx * dy + MB_c[k] * dy * dy);
        U += e;
        gx += e * (2.0 * MB_a[k] * dx + MB_b[k] * dy);
        gy += e * (MB_b[k] * dx + 2.0 * MB_c[k] * dy);
    }
    if (fx) *fx = -gx;
    if (fy) *fy = -gy;
    return U;
}

/* Three-well test landscape in 3-D (a synthetic free-energy surface for the
 * CV-space metadynamics runs that generate long hill lists): three Gaussian
 * wells in a harmonic confinement,
 *   U(r) = -sum_m A_m exp(-|r - c_m|^2 / (2 s_m^2)) + (k/2) |r|^2,
 * A = (8, 6, 7), s = (0.45, 0.40, 0.50), c_1 = (-1, 0, 0),
 * c_2 = (1, 0.2, -0.3), c_3 = (0.1, 1.3, 0.6), k = 1.5.  f[3] = -grad U. */
static const double W3_A[3] = {8.0, 6.0, 7.0};
static const double W3_S[3] = {0.45, 0.40, 0.50};
static const double W3_C[3][3] = {{-1.0, 0.0, 0.0}, {1.0, 0.2, -0.3}, {0.1, 1.3, 0.6}};
static const double W3_K = 1.5;

double orc_wells3(const double* r, double* f)
{
    double U = 0.5 * W3_K * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double g[3] = {W3_K * r[0], W3_K * r[1], W3_K * r[2]};
    for (int m = 0; m < 3; ++m) {
        double d[3] = {r[0] - W3_C[m][0], r[1] - W3_C[m][1], r[2] - W3_C[m][2]};
        double q = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / (2.0 * W3_S[m] * W3_S[m]);
        double e = W3_A[m] * exp(-q);
        U -= e;
        for (int k = 0; k < 3; ++k) g[k] += e * d[k] / (W3_S[m] * W3_S[m]);
    }
    if (f)
        for (int k = 0; k < 3; ++k) f[k] = -g[k];
    return U;
}

/* 12-6 Lennard-Jones, all pairs, minimum image, truncated at rc, energy
 * shifted to zero at rc.  f[n][3] is overwritten.  Returns the energy. */
double orc_lj(int64_t n, const double* x, const double* box, double eps, double sig, double rc, double* f)
{
    double rc2 = rc * rc;
    double sr6c = pow(sig / rc, 6.0);
    double ushift = 4.0 * eps * (sr6c * sr6c - sr6c);
    double U = 0.0;
#pragma omp parallel for reduction(+ : U) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        long double fi[3] = {0.0L, 0.0L, 0.0L}; /* terms of both signs cancel: extended precision */
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            orc_delta(&x[3 * i], &x[3 * j], box, d);
            double r2 = dot3(d, d);
            if (r2 >= rc2) continue;
            double sr2 = sig * sig / r2;
            double sr6 = sr2 * sr2 * sr2;
            double fr = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2; /* -dU/dr / r */
            for (int k = 0; k < 3; ++k) fi[k] += fr * d[k];
            U += 0.5 * (4.0 * eps * (sr6 * sr6 - sr6) - ushift);
        }
        for (int k = 0; k < 3; ++k) f[3 * i + k] = (double)fi[k];
    }
    return U;
}

/* Dihedral angle of four points, IUPAC sign convention:
 * b1 = p1-p0, b2 = p2-p1, b3 = p3-p2, n1 = b1 x b2, n2 = b2 x b3,
 * phi = atan2(|b2| b1.n2, n1.n2) in (-pi, pi]; cis = 0, trans = pi.
 * If g != NULL it receives d phi / d p_k (k = 0..3, 3 components each). */
static double orc_dihedral_pts(const double* p0, const double* p1, const double* p2, const double* p3,
                               const double* box, double g[4][3])
{
    double b1[3], b2[3], b3[3], n1[3], n2[3];
    orc_delta(p1, p0, box, b1);
    orc_delta(p2, p1, box, b2);
    orc_delta(p3, p2, box, b3);
    cross3(b1, b2, n1);
    cross3(b2, b3, n2);
    double nb2 = sqrt(dot3(b2, b2));
    double phi = atan2(nb2 * dot3(b1, n2), dot3(n1, n2));
    if (g) {
        double n1sq = dot3(n1, n1), n2sq = dot3(n2, n2), b2sq = dot3(b2, b2);
        double a = dot3(b1, b2) / b2sq, c = dot3(b3, b2) / b2sq;
        for (int k = 0; k < 3; ++k) {
            g[0][k] = -nb2 / n1sq * n1[k];
            g[3][k] = nb2 / n2sq * n2[k];
        }
        for (int k = 0; k < 3; ++k) {
            g[1][k] = -(1.0 + a) * g[0][k] + c * g[3][k];
            g[2][k] = -(1.0 + c) * g[3][k] + a * g[0][k];
        }
    }
    return phi;
}

/* Bead-chain force field (per chain of nb consecutive beads):
 * bonds k_b/2 (r - r0)^2, angles k_a/2 (theta - theta0)^2,
 * torsions k_t (1 + cos 3 phi).  f is overwritten for the chain's beads. */
double orc_chain(int64_t nb, const double* x, double kb, double r0, double ka, double th0, double kt, double* f)
{
    double U = 0.0;
    for (int64_t i = 0; i < 3 * nb; ++i) f[i] = 0.0;
    for (int64_t i = 0; i + 1 < nb; ++i) {
        double d[3];
        orc_delta(&x[3 * (i + 1)], &x[3 * i], NULL, d);
        double r = sqrt(dot3(d, d));
        U += 0.5 * kb * (r - r0) * (r - r0);
        double c = -kb * (r - r0) / r; /* force on bead i+1 = c * d */
        for (int k = 0; k < 3; ++k) {
            f[3 * (i + 1) + k] += c * d[k];
            f[3 * i + k] -= c * d[k];
        }
    }
    for (int64_t i = 0; i + 2 < nb; ++i) {
        double u[3], v[3];
        orc_delta(&x[3 * i], &x[3 * (i + 1)], NULL, u);      /* bead i   - bead i+1 */
        orc_delta(&x[3 * (i + 2)], &x[3 * (i + 1)], NULL, v); /* bead i+2 - bead i+1 */
        double nu = sqrt(dot3(u, u)), nv = sqrt(dot3(v, v));
        double cs = dot3(u, v) / (nu * nv);
        double th = acos(cs);
        U += 0.5 * ka * (th - th0) * (th - th0);
        /* dtheta/dcos = -1/sin(theta) */
        double dUdcos = ka * (th - th0) * (-1.0 / sin(th));
        for (int k = 0; k < 3; ++k) {
            double dcos_du = v[k] / (nu * nv) - cs * u[k] / (nu * nu);
            double dcos_dv = u[k] / (nu * nv) - cs * v[k] / (nv * nv);
            f[3 * i + k] -= dUdcos * dcos_du;
            f[3 * (i + 2) + k] -= dUdcos * dcos_dv;
            f[3 * (i + 1) + k] += dUdcos * (dcos_du + dcos_dv);
        }
    }
    for (int64_t i = 0; i + 3 < nb; ++i) {
        double g[4][3];
        double phi = orc_dihedral_pts(&x[3 * i], &x[3 * (i + 1)], &x[3 * (i + 2)], &x[3 * (i + 3)], NULL, g);
        U += kt * (1.0 + cos(3.0 * phi));
        double dUdphi = -3.0 * kt * sin(3.0 * phi);
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 3; ++k) f[3 * (i + a) + k] -= dUdphi * g[a][k];
    }
    return U;
}

/* ------------------------------------------------------------------------ */
/* Collective variables (Sec. 2.2).  Each evaluates xi for one walker whose  */
/* atoms are x[0..n-1] and writes the dense Jacobian J[n][3] = d xi / d x.   */
/* ------------------------------------------------------------------------ */
enum {
    ORC_CV_COMPONENT = 1,
    ORC_CV_DIHEDRAL = 2,
    ORC_CV_COORDINATION = 3,
    ORC_CV_RG = 4,
    ORC_CV_QPAIRS = 5,
    ORC_CV_DISTANCE = 6,
    ORC_CV_ANGLE = 7,
    ORC_CV_GYRATION = 8
};
enum { ORC_CV_INTENSIVE = 1 };

typedef struct {
    int64_t kind;
    int64_t n_a;        /* size of group a; -1 = all atoms of the walker */
    const int32_t* a;   /* walker-local indices */
    int64_t n_b;        /* coordination partner group; -1 = all atoms */
    const int32_t* b;
    int64_t axis;       /* Component */
    double r0;          /* switching-function distance */
    int64_t nn, mm;     /* switching-function exponents (mm must be 2 nn) */
    double scale;       /* multiplier; 0 = default (see each CV) */
    int64_t flags;      /* ORC_CV_INTENSIVE */
    double period;      /* > 0: periodic CV with this period */
} orc_cv;

/* Rational switching function s(r) = (1 - x^n) / (1 - x^m), x = r / r0.
 * With m = 2n this equals 1 / (1 + x^n) exactly (the factor 1 - x^n cancels),
 * which also removes the 0/0 at r = r0 (s = 1/2).  Returns s and, through
 * *gr, (ds/dr) / r so that d s / d r_i = gr * (r_i - r_j). */
static double orc_switch(double r2, double r0, int64_t nn, double* gr)
{
    double r = sqrt(r2);
    double x = r / r0;
    double xn = pow(x, (double)nn);
    double s = 1.0 / (1.0 + xn);
    double dsdr = -(double)nn * pow(x, (double)(nn - 1)) / r0 * s * s;
    if (gr) *gr = dsdr / r;
    return s;
}

static int64_t orc_group(int64_t na, const int32_t* a, int64_t n, int64_t k) { return na < 0 ? k : (int64_t)a[k]; }

/* Members of a group unwrapped by the minimum image relative to its first
 * member (u [m][3]) and their mean c: the equal-mass centre used by Rg,
 * Distance and the gyration tensor. */
static void orc_group_unwrap(int64_t na, const int32_t* a, int64_t n, const double* x, const double* box, double* u,
                             double c[3])
{
    int64_t m = na < 0 ? n : na;
    int64_t i0 = orc_group(na, a, n, 0);
    long double cl[3] = {0.0L, 0.0L, 0.0L};
    for (int64_t p = 0; p < m; ++p) {
        int64_t i = orc_group(na, a, n, p);
        double d[3];
        orc_delta(&x[3 * i], &x[3 * i0], box, d);
        for (int k = 0; k < 3; ++k) {
            u[3 * p + k] = x[3 * i0 + k] + d[k];
            cl[k] += u[3 * p + k];
        }
    }
    for (int k = 0; k < 3; ++k) c[k] = (double)(cl[k] / (long double)m);
}

/* Eigenvalues (ascending) and unit eigenvectors (columns of V) of a real
 * symmetric 3x3 matrix by cyclic Jacobi rotations (Golub & Van Loan,
 * Matrix Computations, Sec. 8.5): each rotation zeroes one off-diagonal
 * element; sweeps repeat until the off-diagonal norm is negligible. */
static void orc_eig3(const double S[3][3], double lam[3], double V[3][3])
{
    double A[3][3];
    memcpy(A, S, sizeof(A));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-40 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation angle: tan(2 theta) = 2 A_pq / (A_qq - A_pp) */
                double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < 3; ++k) { /* A <- A G (columns p, q) */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 3; ++k) { /* A <- G^T A (rows p, q) */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 3; ++k) { /* V <- V G */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i) /* sort ascending */
        for (int j = i + 1; j < 3; ++j)
            if (A[idx[j]][idx[j]] < A[idx[i]][idx[i]]) {
                int t = idx[i];
                idx[i] = idx[j];
                idx[j] = t;
            }
    double W[3][3];
    for (int k = 0; k < 3; ++k) {
        lam[k] = A[idx[k]][idx[k]];
        for (int i = 0; i < 3; ++i) W[i][k] = V[i][idx[k]];
    }
    memcpy(V, W, sizeof(W));
}

/* Evaluate one CV for one walker.  Returns 0 or -1 on bad input. */
int orc_cv_eval(const orc_cv* cv, int64_t n, const double* x, const double* box, double* xi, double* J)
{
    /* the switching function is written for m = 2n only (orc_switch): any
     * other exponent pair is refused, not evaluated as something else */
    if ((cv->kind == ORC_CV_COORDINATION || cv->kind == ORC_CV_QPAIRS) && (cv->nn < 1 || cv->mm != 2 * cv->nn))
        return -1;
    for (int64_t i = 0; i < 3 * n; ++i) J[i] = 0.0;
    switch (cv->kind) {
    case ORC_CV_COMPONENT: {
        /* Sec. 2.2 AxisCV "Component": one coordinate of one atom. */
        int64_t i = cv->a[0];
        double sc = cv->scale != 0.0 ? cv->scale : 1.0;
        *xi = sc * x[3 * i + cv->axis];
        J[3 * i + cv->axis] = sc;
        return 0;
    }
    case ORC_CV_DIHEDRAL: {
        /* Sec. 2.2 FourPointCV "DihedralAngle". */
        double g[4][3];
        const int32_t* a = cv->a;
        *xi = orc_dihedral_pts(&x[3 * a[0]], &x[3 * a[1]], &x[3 * a[2]], &x[3 * a[3]], box, g);
        for (int p = 0; p < 4; ++p)
            for (int k = 0; k < 3; ++k) J[3 * a[p] + k] += g[p][k];
        return 0;
    }
    case ORC_CV_COORDINATION: {
        /* Switching-function coordination number (not defined in the paper):
         * xi = scale * sum_{i in A} sum_{j in B, j != i} s(r_ij),
         * default scale = 1/|A| (mean coordination of group A). */
        int64_t na = cv->n_a < 0 ? n : cv->n_a;
        int64_t nb = cv->n_b < 0 ? n : cv->n_b;
        double sc = cv->scale != 0.0 ? cv->scale : 1.0 / (double)na;
        /* sums over up to ~1e7 pair terms accumulate in extended precision
         * so that the reference's own rounding stays far below the parity
         * tolerances */
        long double sum = 0.0L;
        long double* Jl = (long double*)calloc(3 * (size_t)n, sizeof(long double));
        for (int64_t p = 0; p < na; ++p) {
            int64_t i = orc_group(cv->n_a, cv->a, n, p);
            for (int64_t q = 0; q < nb; ++q) {
                int64_t j = orc_group(cv->n_b, cv->b, n, q);
                if (j == i) continue;
                double d[3], gr;
                orc_delta(&x[3 * i], &x[3 * j], box, d);
                sum += orc_switch(dot3(d, d), cv->r0, cv->nn, &gr);
                for (int k = 0; k < 3; ++k) {
                    Jl[3 * i + k] += gr * d[k];
                    Jl[3 * j + k] -= gr * d[k];
                }
            }
        }
        for (int64_t i = 0; i < 3 * n; ++i) J[i] = (double)(sc * Jl[i]);
        free(Jl);
        *xi = (double)(sc * sum);
        return 0;
    }
    case ORC_CV_RG: {
        /* Sec. 2.2 "RadiusofGyration", equal masses:
         * Rg = sqrt(1/m sum_k |u_k - c|^2), u_k = positions unwrapped by the
         * minimum image relative to the group's first atom, c = mean(u).
         * INTENSIVE divides by m^(1/3). */
        int64_t m = cv->n_a < 0 ? n : cv->n_a;
        double* u = (double*)malloc(sizeof(double) * 3 * (size_t)m);
        int64_t i0 = orc_group(cv->n_a, cv->a, n, 0);
        long double cl[3] = {0.0L, 0.0L, 0.0L};
        for (int64_t p = 0; p < m; ++p) {
            int64_t i = orc_group(cv->n_a, cv->a, n, p);
            double d[3];
            orc_delta(&x[3 * i], &x[3 * i0], box, d);
            for (int k = 0; k < 3; ++k) {
                u[3 * p + k] = x[3 * i0 + k] + d[k];
                cl[k] += u[3 * p + k];
            }
        }
        double c[3];
        for (int k = 0; k < 3; ++k) c[k] = (double)(cl[k] / (long double)m);
        long double s2 = 0.0L;
        for (int64_t p = 0; p < m; ++p)
            for (int k = 0; k < 3; ++k) s2 += (u[3 * p + k] - c[k]) * (u[3 * p + k] - c[k]);
        double rg = sqrt((double)(s2 / (long double)m));
        double sc = cv->scale != 0.0 ? cv->scale : 1.0;
        if (cv->flags & ORC_CV_INTENSIVE) sc /= cbrt((double)m);
        for (int64_t p = 0; p < m; ++p) {
            int64_t i = orc_group(cv->n_a, cv->a, n, p);
            for (int k = 0; k < 3; ++k) J[3 * i + k] += sc * (u[3 * p + k] - c[k]) / ((double)m * rg);
        }
        free(u);
        *xi = sc * rg;
        return 0;
    }
    case ORC_CV_DISTANCE: {
        /* Sec. 2.2 TwoPointCV "Distance": distance between the equal-mass
         * centres of groups A and B (each unwrapped relative to its first
         * member), the centre difference taken by the minimum image.
         * dxi/dr = -n/|A| for members of A, +n/|B| for members of B, n the
         * unit vector from c_A to c_B; A and B are disjoint. */
        int64_t ma = cv->n_a, mb = cv->n_b;
        double* ua = (double*)malloc(sizeof(double) * 3 * (size_t)ma);
        double* ub = (double*)malloc(sizeof(double) * 3 * (size_t)mb);
        double ca[3], cb[3], d[3];
        orc_group_unwrap(ma, cv->a, n, x, box, ua, ca);
        orc_group_unwrap(mb, cv->b, n, x, box, ub, cb);
        orc_delta(cb, ca, box, d);
        double r = sqrt(dot3(d, d));
        double sc = cv->scale != 0.0 ? cv->scale : 1.0;
        for (int64_t p = 0; p < ma; ++p)
            for (int k = 0; k < 3; ++k) J[3 * cv->a[p] + k] -= sc * d[k] / r / (double)ma;
        for (int64_t p = 0; p < mb; ++p)
            for (int k = 0; k < 3; ++k) J[3 * cv->b[p] + k] += sc * d[k] / r / (double)mb;
        free(ua);
        free(ub);
        *xi = sc * r;
        return 0;
    }
    case ORC_CV_ANGLE: {
        /* Sec. 2.2 ThreePointCV "Angle" at the middle atom: u = p0 - p1,
         * v = p2 - p1 (minimum image), theta = atan2(|u x v|, u.v) in [0, pi].
         * With w = u x v, s = |w|, c = u.v, w^ = w / s:
         * dtheta/du = (c (v x w^) - s v) / (s^2 + c^2),
         * dtheta/dv = (c (w^ x u) - s u) / (s^2 + c^2),
         * dtheta/dp1 = -(dtheta/du + dtheta/dv).  At 0 and pi (s = 0) the
         * gradient is taken as 0. */
        int64_t i0 = cv->a[0], i1 = cv->a[1], i2 = cv->a[2];
        double u[3], v[3], w[3], wh[3] = {0.0, 0.0, 0.0}, vw[3], wu[3];
        orc_delta(&x[3 * i0], &x[3 * i1], box, u);
        orc_delta(&x[3 * i2], &x[3 * i1], box, v);
        cross3(u, v, w);
        double sn = sqrt(dot3(w, w)), cs = dot3(u, v);
        double th = atan2(sn, cs);
        double sc = cv->scale != 0.0 ? cv->scale : 1.0;
        if (sn > 0.0) {
            for (int k = 0; k < 3; ++k) wh[k] = w[k] / sn;
            cross3(v, wh, vw);
            cross3(wh, u, wu);
            double den = sn * sn + cs * cs;
            for (int k = 0; k < 3; ++k) {
                double gu = (cs * vw[k] - sn * v[k]) / den;
                double gv = (cs * wu[k] - sn * u[k]) / den;
                J[3 * i0 + k] += sc * gu;
                J[3 * i2 + k] += sc * gv;
                J[3 * i1 + k] -= sc * (gu + gv);
            }
        }
        *xi = sc * th;
        return 0;
    }
    case ORC_CV_GYRATION: {
        /* Sec. 2.2 gyration-tensor CVs (AxisCV PrincipalMoment; Asphericity,
         * Acylindricity, ShapeAnisotropy), equal masses.  S = 1/m sum_k
         * (u_k - c)(u_k - c)^T with u, c as for Rg; eigenvalues l1 <= l2 <=
         * l3, unit eigenvectors e1..e3.  axis selects the quantity:
         *   0, 1, 2: l1, l2, l3 (principal moments);
         *   3: asphericity b = l3 - (l1 + l2)/2;
         *   4: acylindricity c = l2 - l1;
         *   5: relative shape anisotropy k2 = 3/2 (l1^2+l2^2+l3^2)/(l1+l2+l3)^2 - 1/2.
         * For a simple eigenvalue dl_j/dr_k = (2/m) (e_j.(u_k - c)) e_j (the
         * centring term sums to zero), and the quantity's gradient is
         * sum_j (dq/dl_j) dl_j/dr_k. */
        int64_t m = cv->n_a < 0 ? n : cv->n_a;
        double* u = (double*)malloc(sizeof(double) * 3 * (size_t)m);
        double c[3];
        orc_group_unwrap(cv->n_a, cv->a, n, x, box, u, c);
        long double Sl[3][3] = {{0.0L}};
        for (int64_t p = 0; p < m; ++p)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Sl[i][j] += (u[3 * p + i] - c[i]) * (u[3 * p + j] - c[j]);
        double S[3][3], lam[3], V[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] = (double)(Sl[i][j] / (long double)m);
        orc_eig3(S, lam, V);
        double q, g[3] = {0.0, 0.0, 0.0};
        double T = lam[0] + lam[1] + lam[2], Q = lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2];
        switch (cv->axis) {
        case 0: case 1: case 2:
            q = lam[cv->axis];
            g[cv->axis] = 1.0;
            break;
        case 3:
            q = lam[2] - 0.5 * (lam[0] + lam[1]);
            g[0] = -0.5;
            g[1] = -0.5;
            g[2] = 1.0;
            break;
        case 4:
            q = lam[1] - lam[0];
            g[0] = -1.0;
            g[1] = 1.0;
            break;
        case 5:
            q = 1.5 * Q / (T * T) - 0.5;
            for (int j = 0; j < 3; ++j) g[j] = 3.0 * (lam[j] * T - Q) / (T * T * T);
            break;
        default:
            free(u);
            return -1;
        }
        double sc = cv->scale != 0.0 ? cv->scale : 1.0;
        for (int64_t p = 0; p < m; ++p) {
            int64_t i = orc_group(cv->n_a, cv->a, n, p);
            for (int j = 0; j < 3; ++j) {
                double proj = 0.0;
                for (int k = 0; k < 3; ++k) proj += V[k][j] * (u[3 * p + k] - c[k]);
                for (int k = 0; k < 3; ++k) J[3 * i + k] += sc * g[j] * 2.0 / (double)m * proj * V[k][j];
            }
        }
        free(u);
        *xi = sc * q;
        return 0;
    }
    case ORC_CV_QPAIRS: {
        /* Q-like pair count (not in the paper): mean switching function over
         * a fixed list of pairs a[2p], a[2p+1]. */
        int64_t np = cv->n_a / 2;
        double sc = cv->scale != 0.0 ? cv->scale : 1.0 / (double)np;
        long double sum = 0.0L;
        long double* Jl = (long double*)calloc(3 * (size_t)n, sizeof(long double));
        for (int64_t p = 0; p < np; ++p) {
            int64_t i = cv->a[2 * p], j = cv->a[2 * p + 1];
            double d[3], gr;
            orc_delta(&x[3 * i], &x[3 * j], box, d);
            sum += orc_switch(dot3(d, d), cv->r0, cv->nn, &gr);
            for (int k = 0; k < 3; ++k) {
                Jl[3 * i + k] += gr * d[k];
                Jl[3 * j + k] -= gr * d[k];
            }
        }
        for (int64_t i = 0; i < 3 * n; ++i) J[i] = (double)(sc * Jl[i]);
        free(Jl);
        *xi = (double)(sc * sum);
        return 0;
    }
    default:
        return -1;
    }
}

/* ------------------------------------------------------------------------ */
/* Metadynamics bias (Sec. 2.1.5)                                            */
/* ------------------------------------------------------------------------ */
/* V(xi) = sum_k w_k exp(-sum_i D_ki^2 / (2 sigma_i^2)), D_ki = xi_i - s_ki
 * (minimum image for periodic CVs), and
 * dV/dxi_i = -sum_k w_k exp(...) D_ki / sigma_i^2.
 * Hills are summed in deposition order.  xi and dV are [P][d]; hills are
 * [H][4] = (s_0, s_1, s_2, w). */
void orc_hills_sum(int64_t d, int64_t P, const double* xi, int64_t H, const double* hills, const double* sigma,
                   const double* period, double* V, double* dV)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        /* extended-precision accumulators: up to 1e6 terms per point */
        long double v = 0.0L, g[3] = {0.0L, 0.0L, 0.0L};
        for (int64_t k = 0; k < H; ++k) {
            double D[3], q = 0.0;
            for (int64_t i = 0; i < d; ++i) {
                D[i] = xi[d * p + i] - hills[4 * k + i];
                if (period && period[i] > 0.0) D[i] -= period[i] * nearbyint(D[i] / period[i]);
                q += D[i] * D[i] / (2.0 * sigma[i] * sigma[i]);
            }
            double e = hills[4 * k + 3] * exp(-q);
            v += e;
            for (int64_t i = 0; i < d; ++i) g[i] -= e * D[i] / (sigma[i] * sigma[i]);
        }
        V[p] = (double)v;
        for (int64_t i = 0; i < d; ++i) dV[d * p + i] = (double)g[i];
    }
}

/* Hill height.  Standard metadynamics keeps it fixed (Sec. 2.1.5); the
 * well-tempered variant scales it with the bias factor gamma (Barducci,
 * Bussi & Parrinello 2008, cited in Sec. 2.1.5; the formula is not printed
 * in the paper): w = w0 exp(-V(s) / (kT (gamma - 1))), i.e. Delta T =
 * (gamma - 1) T.  gamma = 0 or infinite selects the standard method. */
double orc_wt_height(double V, double w0, double kT, double gamma)
{
    if (gamma == 0.0 || isinf(gamma)) return w0;
    return w0 * exp(-V / (kT * (gamma - 1.0)));
}

/* Grid storage of the bias (Sec. 2.1.5, optional grid): cell-centred grid,
 * C order (last CV fastest), every cell gets w exp(-sum D^2/(2 sigma^2)). */
void orc_grid_add(int64_t d, const int64_t* bins, const double* lo, const double* hi, const double* period,
                  const double* sigma, const double* s, double w, double* grid)
{
    int64_t n = 1;
    for (int64_t i = 0; i < d; ++i) n *= bins[i];
#pragma omp parallel for schedule(static)
    for (int64_t cell = 0; cell < n; ++cell) {
        int64_t rem = cell;
        double q = 0.0;
        for (int64_t i = d - 1; i >= 0; --i) {
            int64_t k = rem % bins[i];
            rem /= bins[i];
            double c = lo[i] + ((double)k + 0.5) * (hi[i] - lo[i]) / (double)bins[i];
            double D = c - s[i];
            if (period && period[i] > 0.0) D -= period[i] * nearbyint(D / period[i]);
            q += D * D / (2.0 * sigma[i] * sigma[i]);
        }
        grid[cell] += w * exp(-q);
    }
}

/* Bias and its gradient read from the grid (Sec. 2.1.5: the bias potential
 * kept on a pre-defined grid, trading accuracy for speed).  The paper stores
 * the potential only and says nothing of how forces are taken from it; the
 * reading here:
 *   - nodes are the cell centres c_ik = lo_i + (k + 1/2) dx_i, dx_i =
 *     (hi_i - lo_i) / n_i, holding V;
 *   - the gradient at a node along axis i is the central difference
 *     (V[k+1] - V[k-1]) / (2 dx_i); on a non-periodic axis the end nodes
 *     take the one-sided difference (V[1] - V[0]) / dx_i and
 *     (V[n-1] - V[n-2]) / dx_i; periodic axes wrap node indices mod n_i;
 *   - at a point, u_i = (xi_i - lo_i) / dx_i - 1/2; a periodic axis reduces
 *     u_i into [0, n_i), a non-periodic one clamps it to [0, n_i - 1]
 *     (beyond the outermost nodes the edge values hold); the lower corner is
 *     k_i = floor(u_i) (at most n_i - 2 when non-periodic), t_i = u_i - k_i;
 *   - V(xi) and each dV/dxi_i are multilinear interpolations of the node
 *     values over the 2^d corners, corner weight prod_i (t_i or 1 - t_i).
 * Every axis needs n_i >= 2.  xi and dV are [P][d]. */
static double orc_grid_node(int64_t d, const int64_t* bins, const double* grid, const int64_t* k)
{
    int64_t cell = 0;
    for (int64_t i = 0; i < d; ++i) cell = cell * bins[i] + k[i];
    return grid[cell];
}

static double orc_grid_node_grad(int64_t d, const int64_t* bins, const double* lo, const double* hi,
                                 const double* period, const double* grid, const int64_t* k, int64_t axis)
{
    int64_t n = bins[axis];
    double dx = (hi[axis] - lo[axis]) / (double)n;
    int periodic = period && period[axis] > 0.0;
    int64_t kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
    double span;
    if (periodic) {
        kp[axis] = (k[axis] + 1) % n;
        km[axis] = (k[axis] + n - 1) % n;
        span = 2.0 * dx;
    } else if (k[axis] == 0) {
        kp[axis] = 1;
        span = dx;
    } else if (k[axis] == n - 1) {
        km[axis] = n - 2;
        span = dx;
    } else {
        kp[axis] = k[axis] + 1;
        km[axis] = k[axis] - 1;
        span = 2.0 * dx;
    }
    return (orc_grid_node(d, bins, grid, kp) - orc_grid_node(d, bins, grid, km)) / span;
}

int orc_grid_interp(int64_t d, const int64_t* bins, const double* lo, const double* hi, const double* period,
                    const double* grid, int64_t P, const double* xi, double* V, double* dV)
{
    for (int64_t i = 0; i < d; ++i)
        if (bins[i] < 2) return -1;
    for (int64_t p = 0; p < P; ++p) {
        int64_t k0[3] = {0, 0, 0}, k1[3] = {0, 0, 0};
        double t[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < d; ++i) {
            int64_t n = bins[i];
            double dx = (hi[i] - lo[i]) / (double)n;
            double u = (xi[d * p + i] - lo[i]) / dx - 0.5;
            if (period && period[i] > 0.0) {
                u -= (double)n * floor(u / (double)n);
                if (!(u >= 0.0 && u < (double)n)) u = 0.0; /* rounding at n, or a non-finite / huge xi */
                k0[i] = (int64_t)floor(u);
                k1[i] = (k0[i] + 1) % n;
            } else {
                if (!(u >= 0.0)) u = 0.0; /* below the first node, or not a number */
                if (u > (double)(n - 1)) u = (double)(n - 1);
                k0[i] = (int64_t)floor(u);
                if (k0[i] > n - 2) k0[i] = n - 2;
                k1[i] = k0[i] + 1;
            }
            t[i] = u - (double)k0[i];
        }
        double v = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int64_t corner = 0; corner < ((int64_t)1 << d); ++corner) {
            int64_t k[3] = {0, 0, 0};
            double wgt = 1.0;
            for (int64_t i = 0; i < d; ++i) {
                int upper = (int)((corner >> i) & 1);
                k[i] = upper ? k1[i] : k0[i];
                wgt *= upper ? t[i] : 1.0 - t[i];
            }
            v += wgt * orc_grid_node(d, bins, grid, k);
            for (int64_t i = 0; i < d; ++i) g[i] += wgt * orc_grid_node_grad(d, bins, lo, hi, period, grid, k, i);
        }
        V[p] = v;
        for (int64_t i = 0; i < d; ++i) dV[d * p + i] = g[i];
    }
    return 0;
}

/* Free-energy estimate from the WT bias: A = -(gamma/(gamma-1)) V + C,
 * (standard metadynamics: A = -V + C); C puts the minimum at zero.
 * Meaning of A: Sec. 2.1, Eq. (free-energy). */
void orc_fes(int64_t n, const double* grid, double gamma, double* out)
{
    double f = (gamma == 0.0 || isinf(gamma)) ? -1.0 : -gamma / (gamma - 1.0);
    double mn = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        out[i] = f * grid[i];
        if (out[i] < mn) mn = out[i];
    }
    for (int64_t i = 0; i < n; ++i) out[i] -= mn;
}

/* ------------------------------------------------------------------------ */
/* Whole system: engine + bias + BAOAB + deposition                          */
/* ------------------------------------------------------------------------ */
enum {
    ORC_ENGINE_NONE = 0,
    ORC_ENGINE_MB = 1,
    ORC_ENGINE_LJ = 2,
    ORC_ENGINE_CHAIN = 3,
    ORC_ENGINE_HARMONIC = 4,
    ORC_ENGINE_WELLS3 = 5
};

typedef struct {
    int64_t engine;
    int64_t dims;             /* integrated spatial dimensions: 2 (MB) or 3 */
    int64_t n_walkers;
    const int64_t* walker_off;
    const int64_t* walker_n;
    double box[3];            /* > 0: periodic */
    double dt, friction, mass, kT;
    uint64_t seed;
    double lj_eps, lj_sig, lj_rc;
    double bond_k, bond_r0, angle_k, angle_t0, tors_k;
    double harm_k;
    int64_t n_cv;
    const orc_cv* cv;
    double sigma[3];
    double w0, gamma;
    int64_t stride;
    int64_t hill_cap;
    int64_t grid_bins[3];     /* all zero: no grid */
    double grid_lo[3], grid_hi[3];
    int64_t bias_on;
    int64_t bias_grid;        /* 1: the bias is read from the grid (orc_grid_interp), not summed over hills */
    int64_t bias_harm;        /* 1: harmonic bias about per-walker centres (no hills deposited) */
    double harm_kcv[3];       /* spring constant per CV */
    const double* harm_centre; /* [W][3] window centres */
} orc_sys;

typedef struct {
    double* x;      /* [N][3] */
    double* v;      /* [N][3] */
    double* f;      /* [N][3] total force at x */
    double* hills;  /* [hill_cap][4] */
    int64_t n_hills;
    double* grid;   /* [prod bins] or NULL */
    int64_t step;
    double* xi;     /* [W][3] CVs at x */
    double* V;      /* [W] bias at x (hills before any deposit at this step) */
    double* dV;     /* [W][3] */
    double* xi_sum; /* [W][3] sum of xi over the steps run (harmonic bias) */
    int64_t n_samples;
} orc_state;

static int64_t orc_total_atoms(const orc_sys* s)
{
    int64_t w = s->n_walkers - 1;
    return s->walker_off[w] + s->walker_n[w];
}

static void orc_periods(const orc_sys* s, double* period)
{
    for (int i = 0; i < 3; ++i) period[i] = (i < s->n_cv) ? s->cv[i].period : 0.0;
}

/* Engine force for every walker into f (overwritten). */
static void orc_engine(const orc_sys* s, const double* x, double* f)
{
    int64_t N = orc_total_atoms(s);
    for (int64_t i = 0; i < 3 * N; ++i) f[i] = 0.0;
    for (int64_t w = 0; w < s->n_walkers; ++w) {
        int64_t o = s->walker_off[w], n = s->walker_n[w];
        const double* xw = &x[3 * o];
        double* fw = &f[3 * o];
        switch (s->engine) {
        case ORC_ENGINE_MB:
            for (int64_t i = 0; i < n; ++i) orc_mb(xw[3 * i], xw[3 * i + 1], &fw[3 * i], &fw[3 * i + 1]);
            break;
        case ORC_ENGINE_LJ:
            orc_lj(n, xw, s->box, s->lj_eps, s->lj_sig, s->lj_rc, fw);
            break;
        case ORC_ENGINE_CHAIN:
            orc_chain(n, xw, s->bond_k, s->bond_r0, s->angle_k, s->angle_t0, s->tors_k, fw);
            break;
        case ORC_ENGINE_HARMONIC:
            for (int64_t i = 0; i < 3 * n; ++i) fw[i] = -s->harm_k * xw[i];
            break;
        case ORC_ENGINE_WELLS3:
            for (int64_t i = 0; i < n; ++i) orc_wells3(&xw[3 * i], &fw[3 * i]);
            break;
        default:
            break;
        }
    }
}

/* Bias at x: CVs, then V and dV/dxi from the hills sum over the first H
 * hills (grid == NULL) or from the grid (orc_grid_interp), and
 * f -= J^T dV/dxi for every walker.  xi, V, dV receive the per-walker
 * values. */
static int orc_bias_from(const orc_sys* s, const double* x, const double* hills, int64_t H, const double* grid,
                         double* f, double* xi, double* V, double* dV)
{
    double period[3];
    orc_periods(s, period);
    int64_t d = s->n_cv;
    for (int64_t w = 0; w < s->n_walkers; ++w) {
        int64_t o = s->walker_off[w], n = s->walker_n[w];
        double* J = (double*)malloc(sizeof(double) * 3 * (size_t)n * (size_t)d);
        double xw[3] = {0.0, 0.0, 0.0}, vw, gw[3] = {0.0, 0.0, 0.0};
        for (int64_t c = 0; c < d; ++c)
            if (orc_cv_eval(&s->cv[c], n, &x[3 * o], s->box, &xw[c], &J[3 * n * c]) != 0) {
                free(J);
                return -1;
            }
        if (s->bias_harm) {
            /* Harmonic biasing (Sec. 2.1.1): V = k/2 (xi - xi0)^2 per CV,
             * summed; dV/dxi_c = k_c (xi_c - xi0_c), the difference by the
             * minimum image on periodic CVs.  Each walker has its own centre
             * (one umbrella window per walker, Sec. 2.1.2). */
            vw = 0.0;
            for (int64_t c = 0; c < d; ++c) {
                double D = xw[c] - s->harm_centre[3 * w + c];
                if (period[c] > 0.0) D -= period[c] * nearbyint(D / period[c]);
                vw += 0.5 * s->harm_kcv[c] * D * D;
                gw[c] = s->harm_kcv[c] * D;
            }
        } else if (grid) {
            int64_t bins[3] = {s->grid_bins[0], s->grid_bins[1], s->grid_bins[2]};
            if (orc_grid_interp(d, bins, s->grid_lo, s->grid_hi, period, grid, 1, xw, &vw, gw) != 0) {
                free(J);
                return -1;
            }
        } else {
            orc_hills_sum(d, 1, xw, H, hills, s->sigma, period, &vw, gw);
        }
        for (int64_t c = 0; c < d; ++c)
            for (int64_t i = 0; i < 3 * n; ++i) f[3 * o + i] -= gw[c] * J[3 * n * c + i];
        for (int64_t c = 0; c < 3; ++c) {
            xi[3 * w + c] = xw[c];
            dV[3 * w + c] = c < d ? gw[c] : 0.0;
        }
        V[w] = vw;
        free(J);
    }
    return 0;
}

int orc_bias(const orc_sys* s, const double* x, const double* hills, int64_t H, double* f, double* xi, double* V,
             double* dV)
{
    return orc_bias_from(s, x, hills, H, NULL, f, xi, V, dV);
}

/* The same with the bias read from the grid. */
int orc_bias_grid(const orc_sys* s, const double* x, const double* grid, double* f, double* xi, double* V, double* dV)
{
    return orc_bias_from(s, x, NULL, 0, grid, f, xi, V, dV);
}

/* Total force (engine + bias) at the current positions; fills xi, V, dV.
 * With bias_grid set the bias comes from the grid, and so does the V that
 * sets the next hill's height. */
int orc_forces(const orc_sys* s, orc_state* st)
{
    orc_engine(s, st->x, st->f);
    if (!s->bias_on) return 0;
    if (s->bias_grid) return orc_bias_grid(s, st->x, st->grid, st->f, st->xi, st->V, st->dV);
    return orc_bias(s, st->x, st->hills, st->n_hills, st->f, st->xi, st->V, st->dV);
}

/* n steps of BAOAB Langevin dynamics (Leimkuhler & Matthews 2013):
 *   B: v += dt/2 F/m;  A: x += dt/2 v;  O: v = c1 v + sqrt((1-c1^2) kT/m) R;
 *   A: x += dt/2 v;  forces at the new x (engine + bias);  B: v += dt/2 F/m;
 * c1 = exp(-friction dt).  After a step t (counted from 0) with
 * (t+1) % stride == 0 every walker deposits one hill at s = xi(x_{t+1}) with
 * the height from the bias V(s) of the hills that existed before this step's
 * deposits (walkers in index order); the grid, when present, gets the same
 * Gaussian.  Positions are not wrapped into the box; every distance uses the
 * minimum image.  Returns 0, or -3 when the hill capacity is exceeded. */
int orc_run(const orc_sys* s, orc_state* st, int64_t nsteps)
{
    int64_t N = orc_total_atoms(s);
    double c1 = exp(-s->friction * s->dt);
    double c2 = sqrt((1.0 - c1 * c1) * s->kT / s->mass);
    double half = 0.5 * s->dt;
    double period[3];
    orc_periods(s, period);
    int has_grid = s->grid_bins[0] > 0;
    int rc = 0;
    for (int64_t it = 0; it < nsteps; ++it) {
        int64_t t = st->step;
        for (int64_t i = 0; i < N; ++i) {
            double g[3];
            orc_noise3(s->seed, (uint64_t)t, (uint32_t)i, g);
            for (int64_t k = 0; k < s->dims; ++k) {
                double* x = &st->x[3 * i + k];
                double* v = &st->v[3 * i + k];
                *v += half * st->f[3 * i + k] / s->mass;
                *x += half * (*v);
                *v = c1 * (*v) + c2 * g[k];
                *x += half * (*v);
            }
        }
        if (orc_forces(s, st) != 0) return -1;
        for (int64_t i = 0; i < N; ++i)
            for (int64_t k = 0; k < s->dims; ++k) st->v[3 * i + k] += half * st->f[3 * i + k] / s->mass;
        st->step = t + 1;
        if (s->bias_on && s->bias_harm) {
            /* window statistics: xi at the end of every step */
            for (int64_t w = 0; w < s->n_walkers; ++w)
                for (int c = 0; c < 3; ++c) st->xi_sum[3 * w + c] += st->xi[3 * w + c];
            st->n_samples += 1;
            continue; /* harmonic windows deposit no hills */
        }
        if (s->bias_on && s->stride > 0 && (t + 1) % s->stride == 0) {
            if (st->n_hills + s->n_walkers > s->hill_cap) {
                rc = -3;
                continue;
            }
            for (int64_t w = 0; w < s->n_walkers; ++w) {
                double* h = &st->hills[4 * st->n_hills];
                for (int c = 0; c < 3; ++c) h[c] = c < s->n_cv ? st->xi[3 * w + c] : 0.0;
                h[3] = orc_wt_height(st->V[w], s->w0, s->kT, s->gamma);
                st->n_hills += 1;
                if (has_grid) {
                    int64_t bins[3] = {s->grid_bins[0], s->grid_bins[1], s->grid_bins[2]};
                    orc_grid_add(s->n_cv, bins, s->grid_lo, s->grid_hi, period, s->sigma, h, h[3], st->grid);
                }
            }
        }
    }
    return rc;
}

/* Umbrella integration along a path of windows (Sec. 2.1.2; Kaestner &
 * Thiel's estimate in its lowest order): the mean force of window i is
 * dA/dxi at xi_bar_i = -k (xi_bar_i - xi0_i) (minimum image on periodic
 * CVs), and A along the path of the xi_bar_i, in window order, is the
 * trapezoidal integral A_0 = 0, A_{i+1} = A_i + (g_i + g_{i+1})/2 .
 * (xi_bar_{i+1} - xi_bar_i).  mean_xi, centre and g are [W][3]. */
void orc_umbrella_integrate(int64_t W, int64_t d, const double* mean_xi, const double* centre, const double* k,
                            const double* period, double* g, double* A)
{
    for (int64_t w = 0; w < W; ++w)
        for (int64_t c = 0; c < 3; ++c) {
            double D = 0.0;
            if (c < d) {
                D = mean_xi[3 * w + c] - centre[3 * w + c];
                if (period && period[c] > 0.0) D -= period[c] * nearbyint(D / period[c]);
            }
            g[3 * w + c] = c < d ? -k[c] * D : 0.0;
        }
    A[0] = 0.0;
    for (int64_t w = 0; w + 1 < W; ++w) {
        double dA = 0.0;
        for (int64_t c = 0; c < d; ++c) {
            double step = mean_xi[3 * (w + 1) + c] - mean_xi[3 * w + c];
            if (period && period[c] > 0.0) step -= period[c] * nearbyint(step / period[c]);
            dA += 0.5 * (g[3 * w + c] + g[3 * (w + 1) + c]) * step;
        }
        A[w + 1] = A[w] + dA;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
