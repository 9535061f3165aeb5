/*
 * Plain FP64 CPU oracle for finite-element numerical integration of linear
 * tetrahedra and linear 6-node prisms (Banas, Kruzel, Bielanski, "Finite element
 * numerical integration for first order approximations on multi-core
 * architectures", arXiv 1504.01023).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this code: it
 * exists so that the tests, the smoke check and the CPU-baseline leg of the
 * benchmark can compare the CUDA library against a slow, obviously correct
 * statement of the method. It shares no code, header, table or constant with the
 * CUDA library; its quadrature tables and shape functions are written out here
 * independently.
 *
 * What it computes, per element e (Sec. 2.2, Eqs. sm_local and lv_local):
 *   (A^e)^{rs} = int_{Omega_e} sum_{a,b=0..3} c^{a;b} Phi[a][r] Phi[b][s] dOmega
 *   (b^e)^r    = int_{Omega_e} sum_{a=0..3}   d^a     Phi[a][r]          dOmega
 * with Phi[0][k] = phi_k and Phi[i][k] = d phi_k / d x_i, evaluated by the change
 * of variables to the reference element (Eq. change_of_variables) and Gaussian
 * quadrature (Eq. quadrature), in the step order of Algorithm 1 (Sec. 2.3):
 * read coefficients, read geometry, zero A and b, a first loop over integration
 * points forming the Jacobian terms, vol[Q] and the global derivatives, a second
 * loop forming the coefficients at the points, and a third loop doing the
 * five-nested update of A and the update of b. No loop-invariant hoisting, no
 * symmetry shortcut and no fused arithmetic (compiled with -ffp-contract=off).
 *
 * Readings of the paper (where it is silent):
 *  - Index 0 of c and d means the function value, 1..3 the x,y,z derivatives
 *    (Eq. weak_form); row r is the test function, column s the trial function.
 *  - vol[Q] uses |det J| (Algorithm 1 writes det); det < 0 sets flag bit 1.
 *  - |det J| <= 1e-300 at any point (or a zero LU pivot) makes the element
 *    degenerate: A = 0, b = 0, flag bit 2.
 *  - J^{-1} is obtained by LU factorisation with partial pivoting.
 *  - Poisson: c^{i;j} = delta_ij for i,j >= 1, all other c = 0, d^0 given per
 *    element or per integration point, d^i = 0 (Sec. 4.1 "Poisson" case).
 *  - Reference tetrahedron {xi,eta,zeta >= 0, xi+eta+zeta <= 1}; shape functions
 *    1-xi-eta-zeta, xi, eta, zeta for input vertices 0..3.
 *  - Reference prism = triangle {xi,eta >= 0, xi+eta <= 1} x zeta in [-1,1];
 *    phi_k = lambda_k (1-zeta)/2 (bottom, k=0..2), phi_{k+3} = lambda_k (1+zeta)/2
 *    (top), lambda = (1-xi-eta, xi, eta).
 *
 * The mean-ratio shape quality (oracle_quality) is not in the paper; it restates,
 * in single precision as the kernel decides it, the test that selects elements
 * for the double-precision Jacobian path.
 *
 * Parity unpinned: the diffusion term of non-affine (z-jittered) prisms with
 * per-point coefficients has no closed form. It is pinned only indirectly: by
 * exact agreement with the rational closed forms on affine prisms, exact mass
 * and convection terms, and convergence of the brute-force high-order rules.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TET 0
#define OR_PRISM 1
#define OR_POISSON 0
#define OR_GENERIC 1
#define OR_Q_TET1 0
#define OR_Q_TET4 1
#define OR_Q_PRISM6 2
#define OR_Q_TET_COLLAPSED 3 /* brute-force tensor Gauss rule on the collapsed cube, order n */
#define OR_Q_PRISM_TENSOR 4  /* brute-force Duffy triangle x Gauss-Legendre line, order n */

#define MAXQ 4096

/* ---------------------------------------------------------------------------
 * Gauss-Legendre points on [-1,1] by Newton iteration on P_n (textbook
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}).
 * ------------------------------------------------------------------------- */
static void legendre_pair(int n, double z, double *pn, double *dpn) {
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;                                   /* P_n(z) */
    *dpn = n * (z * p1 - p0) / (z * z - 1.0);   /* P_n'(z) */
}

static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pn, dpn;
        for (int it = 0; it < 100; it++) {
            legendre_pair(n, z, &pn, &dpn);
            double dz = pn / dpn;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        legendre_pair(n, z, &pn, &dpn);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

/* ---------------------------------------------------------------------------
 * Quadrature rules (Sec. 2.3, Eq. quadrature: points xi^Q, weights w^Q).
 * The paper only says "Gaussian"; the rules below are the reading used here.
 * ------------------------------------------------------------------------- */
int oracle_quad_size(int rule, int order) {
    switch (rule) {
    case OR_Q_TET1: return 1;
    case OR_Q_TET4: return 4;
    case OR_Q_PRISM6: return 6;
    case OR_Q_TET_COLLAPSED: return (order > 0 && order * order * order <= MAXQ) ? order * order * order : -1;
    case OR_Q_PRISM_TENSOR: return (order > 0 && order * order * order <= MAXQ) ? order * order * order : -1;
    }
    return -1;
}

int oracle_quad_rule(int rule, int order, double *pts, double *wts) {
    int n = oracle_quad_size(rule, order);
    if (n <= 0) return -1;
    if (rule == OR_Q_TET1) {
        /* centroid of the reference tetrahedron, weight = its volume 1/6 */
        pts[0] = 0.25; pts[1] = 0.25; pts[2] = 0.25;
        wts[0] = 1.0 / 6.0;
    } else if (rule == OR_Q_TET4) {
        /* degree-2 rule: barycentric permutations of (b,a,a,a),
           a = (5 - sqrt 5)/20, b = (5 + 3 sqrt 5)/20, equal weights 1/24 */
        double a = (5.0 - sqrt(5.0)) / 20.0, b = (5.0 + 3.0 * sqrt(5.0)) / 20.0;
        /* point k has barycentric coordinate b on vertex k, a elsewhere;
           (xi,eta,zeta) are the barycentric weights of vertices 1,2,3 */
        double bary[4][4] = {{b, a, a, a}, {a, b, a, a}, {a, a, b, a}, {a, a, a, b}};
        for (int q = 0; q < 4; q++) {
            pts[3 * q + 0] = bary[q][1];
            pts[3 * q + 1] = bary[q][2];
            pts[3 * q + 2] = bary[q][3];
            wts[q] = 1.0 / 24.0;
        }
    } else if (rule == OR_Q_PRISM6) {
        /* triangle 3-point rule {(1/6,1/6),(2/3,1/6),(1/6,2/3)}, weights 1/6,
           times the 2-point Gauss-Legendre rule zeta = -+1/sqrt 3, weights 1 */
        double tri[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
        double zl[2] = {-1.0 / sqrt(3.0), 1.0 / sqrt(3.0)};
        int q = 0;
        for (int l = 0; l < 2; l++)
            for (int t = 0; t < 3; t++) {
                pts[3 * q + 0] = tri[t][0];
                pts[3 * q + 1] = tri[t][1];
                pts[3 * q + 2] = zl[l];
                wts[q] = 1.0 / 6.0;
                q++;
            }
    } else if (rule == OR_Q_TET_COLLAPSED) {
        /* collapsed (Duffy) cube: xi = u, eta = v (1-u), zeta = t (1-u)(1-v),
           Jacobian (1-u)^2 (1-v); Gauss-Legendre in u, v, t mapped to [0,1] */
        double gx[64], gw[64];
        if (order > 64) return -1;
        gauss_legendre(order, gx, gw);
        int q = 0;
        for (int i = 0; i < order; i++)
            for (int j = 0; j < order; j++)
                for (int k = 0; k < order; k++) {
                    double u = 0.5 * (gx[i] + 1.0), v = 0.5 * (gx[j] + 1.0), t = 0.5 * (gx[k] + 1.0);
                    pts[3 * q + 0] = u;
                    pts[3 * q + 1] = v * (1.0 - u);
                    pts[3 * q + 2] = t * (1.0 - u) * (1.0 - v);
                    wts[q] = 0.125 * gw[i] * gw[j] * gw[k] * (1.0 - u) * (1.0 - u) * (1.0 - v);
                    q++;
                }
    } else if (rule == OR_Q_PRISM_TENSOR) {
        /* collapsed square for the triangle: xi = u, eta = v (1-u), Jacobian (1-u);
           Gauss-Legendre in zeta on [-1,1] */
        double gx[64], gw[64];
        if (order > 64) return -1;
        gauss_legendre(order, gx, gw);
        int q = 0;
        for (int i = 0; i < order; i++)
            for (int j = 0; j < order; j++)
                for (int k = 0; k < order; k++) {
                    double u = 0.5 * (gx[i] + 1.0), v = 0.5 * (gx[j] + 1.0);
                    pts[3 * q + 0] = u;
                    pts[3 * q + 1] = v * (1.0 - u);
                    pts[3 * q + 2] = gx[k];
                    wts[q] = 0.25 * gw[i] * gw[j] * gw[k] * (1.0 - u);
                    q++;
                }
    }
    return n;
}

/* ---------------------------------------------------------------------------
 * Reference shape functions and their local derivatives (Sec. 2.3, input list:
 * "values of shape functions and their local derivatives", computed on the fly).
 * ------------------------------------------------------------------------- */
static void tet_shape(const double *xi, double *phi, double dphi[][3]) {
    phi[0] = 1.0 - xi[0] - xi[1] - xi[2];
    phi[1] = xi[0];
    phi[2] = xi[1];
    phi[3] = xi[2];
    double d[4][3] = {{-1.0, -1.0, -1.0}, {1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
    memcpy(dphi, d, sizeof d);
}

static void prism_shape(const double *xi, double *phi, double dphi[][3]) {
    double lam[3] = {1.0 - xi[0] - xi[1], xi[0], xi[1]};
    double dlam[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
    double zb = 0.5 * (1.0 - xi[2]), zt = 0.5 * (1.0 + xi[2]);
    for (int k = 0; k < 3; k++) {
        phi[k] = lam[k] * zb;
        phi[k + 3] = lam[k] * zt;
        dphi[k][0] = dlam[k][0] * zb;
        dphi[k][1] = dlam[k][1] * zb;
        dphi[k][2] = -0.5 * lam[k];
        dphi[k + 3][0] = dlam[k][0] * zt;
        dphi[k + 3][1] = dlam[k][1] * zt;
        dphi[k + 3][2] = 0.5 * lam[k];
    }
}

/* ---------------------------------------------------------------------------
 * 3x3 LU factorisation with partial pivoting: det and inverse.
 * Returns 0 on success, -1 on a zero pivot.
 * ------------------------------------------------------------------------- */
static int lu_det_inverse(const double Jin[3][3], double *det, double inv[3][3]) {
    double a[3][3];
    int perm[3] = {0, 1, 2};
    double sign = 1.0;
    memcpy(a, Jin, sizeof a);
    for (int k = 0; k < 3; k++) {
        int p = k;
        for (int i = k + 1; i < 3; i++)
            if (fabs(a[i][k]) > fabs(a[p][k])) p = i;
        if (a[p][k] == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < 3; j++) {
                double t = a[k][j];
                a[k][j] = a[p][j];
                a[p][j] = t;
            }
            int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
            sign = -sign;
        }
        for (int i = k + 1; i < 3; i++) {
            a[i][k] = a[i][k] / a[k][k];
            for (int j = k + 1; j < 3; j++) a[i][j] = a[i][j] - a[i][k] * a[k][j];
        }
    }
    *det = sign * a[0][0] * a[1][1] * a[2][2];
    /* solve J X = I column by column: P J = L U */
    for (int c = 0; c < 3; c++) {
        double y[3];
        for (int i = 0; i < 3; i++) {
            double rhs = (perm[i] == c) ? 1.0 : 0.0;
            for (int j = 0; j < i; j++) rhs = rhs - a[i][j] * y[j];
            y[i] = rhs;
        }
        for (int i = 2; i >= 0; i--) {
            double s = y[i];
            for (int j = i + 1; j < 3; j++) s = s - a[i][j] * inv[j][c];
            inv[i][c] = s / a[i][i];
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 for one element. coords: NS x 3 vertex coordinates.
 * coefs: Poisson -> d^0 (1 value, or NQ values if coef_per_q);
 *        generic -> 20 values C[4][4] row-major then D[4] (or NQ blocks of 20).
 * ------------------------------------------------------------------------- */
static uint8_t integrate_one(int elem_type, int kind, int nq, const double *pts, const double *wts,
                             int coef_per_q, const double *x, const double *coefs, double *Aout,
                             double *bout) {
    const int NS = (elem_type == OR_TET) ? 4 : 6;
    const int ND = 3;
    static const int MAXS = 6;
    uint8_t flags = 0;
    /* storage per integration point, as the algorithm keeps vol[iQ], phi[iD][iS][iQ],
       c[iD][jD][iQ] and d[iD][iQ] */
    double *vol = (double *)malloc(sizeof(double) * nq);
    double *phi = (double *)malloc(sizeof(double) * (ND + 1) * MAXS * nq);
    double *c = (double *)malloc(sizeof(double) * (ND + 1) * (ND + 1) * nq);
    double *d = (double *)malloc(sizeof(double) * (ND + 1) * nq);
#define PHI(iD, iS, iQ) phi[((iD) * MAXS + (iS)) * nq + (iQ)]
#define CC(iD, jD, iQ) c[((iD) * (ND + 1) + (jD)) * nq + (iQ)]
#define DD(iD, iQ) d[(iD) * nq + (iQ)]
    double A[6][6], b[6];
    int degenerate = 0;

    /* initialize A^e and b^e */
    for (int r = 0; r < NS; r++) {
        b[r] = 0.0;
        for (int s = 0; s < NS; s++) A[r][s] = 0.0;
    }

    /* loop 1 over integration points: Jacobian terms, vol, global derivatives */
    for (int iQ = 0; iQ < nq; iQ++) {
        double phat[6], dphat[6][3];
        if (elem_type == OR_TET)
            tet_shape(&pts[3 * iQ], phat, dphat);
        else
            prism_shape(&pts[3 * iQ], phat, dphat);
        double J[3][3];
        for (int i = 0; i < 3; i++)
            for (int m = 0; m < 3; m++) {
                double s = 0.0;
                for (int k = 0; k < NS; k++) s = s + x[3 * k + i] * dphat[k][m];
                J[i][m] = s;
            }
        double det, inv[3][3];
        if (lu_det_inverse(J, &det, inv) != 0 || !(fabs(det) > 1e-300)) {
            degenerate = 1;
            vol[iQ] = 0.0;
            for (int iD = 0; iD <= ND; iD++)
                for (int iS = 0; iS < NS; iS++) PHI(iD, iS, iQ) = 0.0;
            continue;
        }
        if (det < 0.0) flags |= 2;
        vol[iQ] = fabs(det) * wts[iQ];
        for (int iS = 0; iS < NS; iS++) {
            PHI(0, iS, iQ) = phat[iS];
            for (int i = 0; i < 3; i++) {
                double s = 0.0;
                for (int m = 0; m < 3; m++) s = s + dphat[iS][m] * inv[m][i];
                PHI(1 + i, iS, iQ) = s;
            }
        }
    }

    /* loop 2 over integration points: coefficients c and d */
    for (int iQ = 0; iQ < nq; iQ++) {
        if (kind == OR_POISSON) {
            for (int iD = 0; iD <= ND; iD++) {
                for (int jD = 0; jD <= ND; jD++) CC(iD, jD, iQ) = (iD == jD && iD >= 1) ? 1.0 : 0.0;
                DD(iD, iQ) = 0.0;
            }
            DD(0, iQ) = coef_per_q ? coefs[iQ] : coefs[0];
        } else {
            const double *cq = coef_per_q ? &coefs[20 * iQ] : coefs;
            for (int iD = 0; iD <= ND; iD++) {
                for (int jD = 0; jD <= ND; jD++) CC(iD, jD, iQ) = cq[4 * iD + jD];
                DD(iD, iQ) = cq[16 + iD];
            }
        }
    }

    /* loop 3: the five-nested update of A^e and the update of b^e */
    for (int iQ = 0; iQ < nq; iQ++) {
        for (int iS = 0; iS < NS; iS++) {
            for (int jS = 0; jS < NS; jS++) {
                for (int iD = 0; iD <= ND; iD++) {
                    for (int jD = 0; jD <= ND; jD++) {
                        A[iS][jS] = A[iS][jS] + vol[iQ] * CC(iD, jD, iQ) * PHI(iD, iS, iQ) * PHI(jD, jS, iQ);
                    }
                }
            }
            for (int iD = 0; iD <= ND; iD++) {
                b[iS] = b[iS] + vol[iQ] * DD(iD, iQ) * PHI(iD, iS, iQ);
            }
        }
    }

    /* store the whole A^e and b^e */
    for (int r = 0; r < NS; r++) {
        bout[r] = degenerate ? 0.0 : b[r];
        for (int s = 0; s < NS; s++) Aout[r * NS + s] = degenerate ? 0.0 : A[r][s];
    }
    if (degenerate) flags = 4;
    free(vol);
    free(phi);
    free(c);
    free(d);
#undef PHI
#undef CC
#undef DD
    return flags;
}

/*
 * Integrate n_elem elements of one type (Algorithm 1's element loop).
 * coords  : [n_elem][NS][3] doubles.
 * coefs   : Poisson [n_elem][1 or NQ]; generic [n_elem][1 or NQ][20].
 * A, b    : [n_elem][NS][NS], [n_elem][NS].
 * flags   : [n_elem] bytes (may be NULL): bit1 det<0, bit2 degenerate.
 * Returns 0, or -1 on a bad argument.
 */
int oracle_integrate(int elem_type, int kind, int rule, int order, int coef_per_q, int64_t n_elem,
                     const double *coords, const double *coefs, double *A, double *b, uint8_t *flags,
                     int n_threads) {
    if (elem_type != OR_TET && elem_type != OR_PRISM) return -1;
    if (kind != OR_POISSON && kind != OR_GENERIC) return -1;
    int nq = oracle_quad_size(rule, order);
    if (nq <= 0) return -1;
    int tet_rule = (rule == OR_Q_TET1 || rule == OR_Q_TET4 || rule == OR_Q_TET_COLLAPSED);
    if ((elem_type == OR_TET) != tet_rule) return -1;
    if (coef_per_q && (rule == OR_Q_TET_COLLAPSED || rule == OR_Q_PRISM_TENSOR)) return -1;
    double *pts = (double *)malloc(sizeof(double) * 3 * nq);
    double *wts = (double *)malloc(sizeof(double) * nq);
    oracle_quad_rule(rule, order, pts, wts);
    const int NS = (elem_type == OR_TET) ? 4 : 6;
    const int ncoef = (kind == OR_POISSON ? 1 : 20) * (coef_per_q ? nq : 1);
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int64_t e = 0; e < n_elem; e++) {
        uint8_t f = integrate_one(elem_type, kind, nq, pts, wts, coef_per_q, &coords[e * NS * 3],
                                  &coefs[e * ncoef], &A[e * NS * NS], &b[e * NS]);
        if (flags) flags[e] = f;
    }
    free(pts);
    free(wts);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Coefficients computed at the integration points by a problem-dependent
 * function (Sec. 2.3, input list: "problem dependent parameters that are used
 * for computing coefficients"; Sec. 3.1: the coefficients may come from a
 * special, problem dependent function). The function here is the one the
 * library offers: with u_Q = sum_k phi_k(xi_Q) u_k the value at point Q of a
 * field given by its nodal values u_k, coefficient j (C[4][4] row-major then
 * D[4]) is P[0][j] + P[1][j] u_Q + P[2][j] u_Q^2. Writes the per-point
 * coefficients oracle_integrate takes: generic [n][NQ][20], Poisson [n][NQ]
 * (its d^0, slot 16 of P).
 * ------------------------------------------------------------------------- */
int oracle_coefs_from_u(int elem_type, int kind, int rule, int64_t n_elem, const double *u, const double *P,
                        double *coefs) {
    if (elem_type != OR_TET && elem_type != OR_PRISM) return -1;
    if (kind != OR_POISSON && kind != OR_GENERIC) return -1;
    if (rule != OR_Q_TET1 && rule != OR_Q_TET4 && rule != OR_Q_PRISM6) return -1;
    if ((elem_type == OR_TET) != (rule != OR_Q_PRISM6)) return -1;
    const int nq = oracle_quad_size(rule, 0);
    double pts[3 * 16], wts[16];
    oracle_quad_rule(rule, 0, pts, wts);
    const int NS = (elem_type == OR_TET) ? 4 : 6;
    for (int64_t e = 0; e < n_elem; e++) {
        for (int q = 0; q < nq; q++) {
            double phi[6], dphi[6][3];
            if (elem_type == OR_TET)
                tet_shape(&pts[3 * q], phi, dphi);
            else
                prism_shape(&pts[3 * q], phi, dphi);
            double uq = 0.0;
            for (int k = 0; k < NS; k++) uq = uq + phi[k] * u[e * NS + k];
            if (kind == OR_POISSON) {
                coefs[e * nq + q] = P[16] + P[20 + 16] * uq + P[40 + 16] * uq * uq;
            } else {
                for (int j = 0; j < 20; j++) coefs[(e * nq + q) * 20 + j] = P[j] + P[20 + j] * uq + P[40 + j] * uq * uq;
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Mean-ratio shape quality in single precision (not in the paper).
 * q = 3 |det T|^{2/3} / ||T||_F^2 with T = J S^{-1}, where S maps the reference
 * element onto its ideal: the unit-edge equilateral tetrahedron, or the prism of
 * a unit-edge equilateral triangle and unit height. Edge vectors x_k - x_0 are
 * formed in double and narrowed; everything after that is float. Prisms take the
 * minimum over the six PRISM6 points.
 * ------------------------------------------------------------------------- */
static float quality_from_J(const float J[3][3], const float Sinv[3][3]) {
    float T[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            float s = 0.0f;
            for (int k = 0; k < 3; k++) s = s + J[i][k] * Sinv[k][j];
            T[i][j] = s;
        }
    float det = T[0][0] * (T[1][1] * T[2][2] - T[1][2] * T[2][1]) -
                T[0][1] * (T[1][0] * T[2][2] - T[1][2] * T[2][0]) +
                T[0][2] * (T[1][0] * T[2][1] - T[1][1] * T[2][0]);
    float fro = 0.0f;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) fro = fro + T[i][j] * T[i][j];
    float ad = fabsf(det);
    return 3.0f * cbrtf(ad * ad) / fro;
}

int oracle_quality(int elem_type, int64_t n_elem, const double *coords, float *q, int n_threads) {
    if (elem_type != OR_TET && elem_type != OR_PRISM) return -1;
    /* S^{-1} for the equilateral tetrahedron with vertices (0,0,0), (1,0,0),
       (1/2, sqrt3/2, 0), (1/2, sqrt3/6, sqrt(2/3)): columns of S are those edges */
    double S[3][3] = {{1.0, 0.5, 0.5}, {0.0, sqrt(3.0) / 2.0, sqrt(3.0) / 6.0}, {0.0, 0.0, sqrt(2.0 / 3.0)}};
    if (elem_type == OR_PRISM) {
        double Sp[3][3] = {{1.0, 0.5, 0.0}, {0.0, sqrt(3.0) / 2.0, 0.0}, {0.0, 0.0, 0.5}};
        memcpy(S, Sp, sizeof S);
    }
    double det, Sinvd[3][3];
    lu_det_inverse(S, &det, Sinvd);
    float Sinv[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Sinv[i][j] = (float)Sinvd[i][j];
    double pts[18], wts[6];
    oracle_quad_rule(OR_Q_PRISM6, 0, pts, wts);
    const int NS = (elem_type == OR_TET) ? 4 : 6;
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int64_t e = 0; e < n_elem; e++) {
        const double *x = &coords[e * NS * 3];
        float rel[6][3];
        for (int k = 0; k < NS; k++)
            for (int i = 0; i < 3; i++) rel[k][i] = (float)(x[3 * k + i] - x[i]);
        float qmin;
        if (elem_type == OR_TET) {
            float J[3][3];
            for (int i = 0; i < 3; i++)
                for (int m = 0; m < 3; m++) J[i][m] = rel[m + 1][i];
            qmin = quality_from_J(J, Sinv);
        } else {
            qmin = 1e30f;
            for (int iQ = 0; iQ < 6; iQ++) {
                double phat[6], dphat[6][3];
                prism_shape(&pts[3 * iQ], phat, dphat);
                float J[3][3];
                for (int i = 0; i < 3; i++)
                    for (int m = 0; m < 3; m++) {
                        float s = 0.0f;
                        for (int k = 0; k < 6; k++) s = s + rel[k][i] * (float)dphat[k][m];
                        J[i][m] = s;
                    }
                float qq = quality_from_J(J, Sinv);
                if (!(qq >= qmin)) qmin = qq;
            }
        }
        q[e] = qmin;
    }
    return 0;
}
