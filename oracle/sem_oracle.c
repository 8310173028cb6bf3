/*
 * sem_oracle.c -- plain, slow, FP64 CPU oracle for the spectral-element (SEM)
 * hot path: GLL quadrature, the GLL derivative matrix, trilinear hexahedral
 * geometry, the matrix-free Helmholtz/Poisson operator (ax_helm), the
 * gather-scatter direct-stiffness sum (dssum), the Jacobi diagonal, Jacobi
 * PCG, the 3/2-rule dealiased convective term and a BDF3/EXT3 P_N-P_N
 * Taylor-Green vortex step with kinetic-energy / enstrophy diagnostics.
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library; the two meet only through seeded
 * input arrays.
 *
 * The paper (Chen, Muensch, Iakymchuk, "Mixed-Precision SEM-Based CFD
 * Simulations on GPUs: A Taylor-Green Vortex case") names these components
 * -- ax_helm and tnsr3d (Sec. 2, Fig. 4; Sec. 4, Table 2 rows B-5..B-7),
 * glsc3 (Sec. 2, Fig. 4), gather/scatter and CG+Jacobi (Sec. 1.1, Sec. 2),
 * the TGV case (Sec. 3, Eqs. 1-4) and the accuracy metrics (Sec. 4.2,
 * Eqs. 5-9) -- but prints no SEM formula.  Every SEM definition below is
 * therefore the textbook one (Deville, Fischer & Mund, "High-Order Methods
 * for Incompressible Fluid Flow", 2002, ch. 2-4 and 6), written out plainly
 * in FP64 with no blocking, fusion or reordering beyond the sum-factorised
 * application of a tensor-product matrix.
 *
 * Layouts used here (the oracle's own):
 *   E-vector  u[e][k][j][i], i fastest, e = ex + nelx*(ey + nely*ez)
 *   G         G[c][n] with c = 0..5 -> (11,22,33,12,13,23), n = local node
 *   J^{-1}    jinv[a*3+c][n] = d r_a / d x_c
 *   coords    xyz[c][n]
 *   vertices  vert[((K*(nely+1)+J)*(nelx+1)+I)*3 + c]
 *
 * Reductions are deterministic for any thread count: per-element partial
 * sums are added serially in element order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_BAD_MESH -4
#define ORC_ERR_NOT_CONVERGED -5
#define ORC_ERR_BREAKDOWN -6

#define ORC_NMAX 15

/* Number of OpenMP threads the oracle runs with. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the OpenMP thread count of later calls (n >= 1; timing only). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1-D polynomial tools                                                      */
/* ------------------------------------------------------------------------ */

/* Legendre P_n(x) and P_n'(x) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},  P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre(int n, double x, double *p, double *dp)
{
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        double d2 = d0 + (2.0 * k + 1.0) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    *p = p1; *dp = d1;
}

/* GLL nodes and weights (textbook; the paper's SEM basis, Sec. 1, Sec. 2).
 * xi_0 = -1, xi_N = 1, interior nodes are the roots of P_N'.  Newton on P_N'
 * using P_N'' from the Legendre ODE (1-x^2)P'' = 2xP' - N(N+1)P, started at
 * the Chebyshev-Gauss-Lobatto points -cos(pi i/N), then symmetrised.
 * Weights w_i = 2 / (N(N+1) P_N(xi_i)^2). */
int orc_gll(int N, double *xi, double *w)
{
    if (N < 1 || N > 64) return ORC_ERR_ARG;
    xi[0] = -1.0; xi[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        double x = -cos(M_PI * i / N);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(N, x, &p, &dp);
            double d2p = (2.0 * x * dp - N * (N + 1.0) * p) / (1.0 - x * x);
            double dx = dp / d2p;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xi[i] = x;
    }
    for (int i = 0; i <= N / 2; ++i) {
        double s = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -s; xi[N - i] = s;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int i = 0; i <= N; ++i) {
        double p, dp;
        legendre(N, xi[i], &p, &dp);
        w[i] = 2.0 / (N * (N + 1.0) * p * p);
    }
    return ORC_OK;
}

/* Gauss-Legendre points (roots of P_M) and weights 2 / ((1-x^2) P_M'(x)^2);
 * the over-integration grid of the dealiased convective term. */
int orc_gl(int M, double *eta, double *w)
{
    if (M < 1 || M > 128) return ORC_ERR_ARG;
    for (int q = 0; q < M; ++q) {
        double x = -cos(M_PI * (q + 0.75) / (M + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(M, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        eta[q] = x;
    }
    for (int q = 0; q < M / 2; ++q) {
        double s = 0.5 * (eta[M - 1 - q] - eta[q]);
        eta[q] = -s; eta[M - 1 - q] = s;
    }
    if (M % 2 == 1) eta[M / 2] = 0.0;
    for (int q = 0; q < M; ++q) {
        double p, dp;
        legendre(M, eta[q], &p, &dp);
        w[q] = 2.0 / ((1.0 - eta[q] * eta[q]) * dp * dp);
    }
    return ORC_OK;
}

/* GLL derivative matrix D_ij = l_j'(xi_i), D[i*(N+1)+j] (textbook closed
 * form): D_ij = P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j)) for i != j; the
 * diagonal is minus the row's off-diagonal sum, which equals the closed form
 * (D_00 = -N(N+1)/4, D_NN = N(N+1)/4, 0 otherwise) up to rounding and makes
 * D*1 = 0 hold to rounding. */
int orc_deriv(int N, const double *xi, double *D)
{
    if (N < 1 || N > 64) return ORC_ERR_ARG;
    int n = N + 1;
    double P[65];
    for (int i = 0; i < n; ++i) { double dp; legendre(N, xi[i], &P[i], &dp); }
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            D[i * n + j] = P[i] / (P[j] * (xi[i] - xi[j]));
            s += D[i * n + j];
        }
        D[i * n + i] = -s;
    }
    return ORC_OK;
}

/* Lagrange interpolation matrix from the N+1 GLL nodes to M points x:
 * J[q*(N+1)+j] = l_j(x_q) = prod_{k != j} (x_q - xi_k) / (xi_j - xi_k). */
int orc_interp(int N, const double *xi, int M, const double *x, double *J)
{
    int n = N + 1;
    for (int q = 0; q < M; ++q)
        for (int j = 0; j < n; ++j) {
            double l = 1.0;
            for (int k = 0; k < n; ++k)
                if (k != j) l *= (x[q] - xi[k]) / (xi[j] - xi[k]);
            J[q * n + j] = l;
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Trilinear hexahedral geometry                                             */
/* ------------------------------------------------------------------------ */

static void elem_vertices(int nelx, int nely, int e, const double *vert, double X[8][3])
{
    int ex = e % nelx, ey = (e / nelx) % nely, ez = e / (nelx * nely);
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                size_t vi = ((size_t)(ez + c) * (nely + 1) + (ey + b)) * (nelx + 1) + (ex + a);
                for (int d = 0; d < 3; ++d) X[a + 2 * b + 4 * c][d] = vert[vi * 3 + d];
            }
}

/* x(r,s,t) = sum_{abc} X_abc phi_a(r) phi_b(s) phi_c(t), phi_0 = (1-r)/2,
 * phi_1 = (1+r)/2; jac[d][a] = d x_d / d r_a. */
static void trilinear(const double X[8][3], double r, double s, double t,
                      double x[3], double jac[3][3])
{
    double pr[2] = {0.5 * (1 - r), 0.5 * (1 + r)}, dr[2] = {-0.5, 0.5};
    double ps[2] = {0.5 * (1 - s), 0.5 * (1 + s)}, ds[2] = {-0.5, 0.5};
    double pt[2] = {0.5 * (1 - t), 0.5 * (1 + t)}, dt[2] = {-0.5, 0.5};
    for (int d = 0; d < 3; ++d) {
        x[d] = 0; jac[d][0] = jac[d][1] = jac[d][2] = 0;
    }
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const double *v = X[a + 2 * b + 4 * c];
                for (int d = 0; d < 3; ++d) {
                    x[d] += v[d] * pr[a] * ps[b] * pt[c];
                    jac[d][0] += v[d] * dr[a] * ps[b] * pt[c];
                    jac[d][1] += v[d] * pr[a] * ds[b] * pt[c];
                    jac[d][2] += v[d] * pr[a] * ps[b] * dt[c];
                }
            }
}

/* det and inverse of a 3x3 matrix by cofactors: inv[a][d] = (jac^{-1})_{ad}. */
static double inv3(const double m[3][3], double inv[3][3])
{
    double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
    return det;
}

/* Node coordinates, J^{-1}, the six geometric factors and the mass
 * (pre-processing "geometry" of the P_N-P_N step, Sec. 1.1 Fig. 3):
 *   B    = w_i w_j w_k |J|
 *   G_ab = w_i w_j w_k |J| sum_c (dr_a/dx_c)(dr_b/dx_c),
 *          (a,b) in {11,22,33,12,13,23}.
 * Any output pointer may be NULL.  Returns ORC_ERR_BAD_MESH if some |J| <= 0. */
int orc_geom(int N, int nelx, int nely, int nelz, const double *vert,
             double *xyz, double *jinv, double *G, double *B)
{
    if (N < 1 || N > ORC_NMAX || nelx < 1 || nely < 1 || nelz < 1) return ORC_ERR_ARG;
    int n = N + 1, n3 = n * n * n;
    long E = (long)nelx * nely * nelz;
    size_t nL = (size_t)E * n3;
    double xi[ORC_NMAX + 1], w[ORC_NMAX + 1];
    orc_gll(N, xi, w);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long e = 0; e < E; ++e) {
        double X[8][3];
        elem_vertices(nelx, nely, (int)e, vert, X);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    size_t p = (size_t)e * n3 + (size_t)(k * n + j) * n + i;
                    double x[3], jac[3][3], inv[3][3];
                    trilinear(X, xi[i], xi[j], xi[k], x, jac);
                    double det = inv3(jac, inv);
                    if (!(det > 0)) bad = 1;
                    double wq = w[i] * w[j] * w[k] * det;
                    if (xyz)
                        for (int c = 0; c < 3; ++c) xyz[c * nL + p] = x[c];
                    if (jinv)
                        for (int a = 0; a < 3; ++a)
                            for (int c = 0; c < 3; ++c) jinv[(a * 3 + c) * nL + p] = inv[a][c];
                    if (B) B[p] = wq;
                    if (G) {
                        static const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
                        for (int g = 0; g < 6; ++g) {
                            double s = 0;
                            for (int c = 0; c < 3; ++c) s += inv[pa[g]][c] * inv[pb[g]][c];
                            G[g * nL + p] = wq * s;
                        }
                    }
                }
    }
    return bad ? ORC_ERR_BAD_MESH : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Element operator (ax_helm: Sec. 4 Table 2 rows B-6/B-7)                   */
/* ------------------------------------------------------------------------ */

/* Gradient in reference space of one element field u (n^3):
 * ur = (I x I x D) u, us = (I x D x I) u, ut = (D x I x I) u. */
static void ref_grad(int n, const double *D, const double *u, double *ur, double *us, double *ut)
{
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double a = 0, b = 0, c = 0;
                for (int l = 0; l < n; ++l) {
                    a += D[i * n + l] * u[(k * n + j) * n + l];
                    b += D[j * n + l] * u[(k * n + l) * n + i];
                    c += D[k * n + l] * u[(l * n + j) * n + i];
                }
                int p = (k * n + j) * n + i;
                ur[p] = a; us[p] = b; ut[p] = c;
            }
}

/* out += (I x I x D^T) vr + (I x D^T x I) vs + (D^T x I x I) vt. */
static void ref_grad_T(int n, const double *D, const double *vr, const double *vs,
                       const double *vt, double *out)
{
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double s = 0;
                for (int l = 0; l < n; ++l) {
                    s += D[l * n + i] * vr[(k * n + j) * n + l];
                    s += D[l * n + j] * vs[(k * n + l) * n + i];
                    s += D[l * n + k] * vt[(l * n + j) * n + i];
                }
                out[(k * n + j) * n + i] += s;
            }
}

/* w_e = h1 (D^T G D) u_e + h2 B u_e on every element (local, not assembled):
 *   u_a = D_a u,  v_a = h1 sum_b G_ab u_b,  w = sum_a D_a^T v_a + h2 B u. */
int orc_ax(int N, long E, const double *D, const double *G, const double *B,
           double h1, double h2, const double *u, double *w)
{
    if (N < 1 || N > ORC_NMAX || E < 0) return ORC_ERR_ARG;
    int n = N + 1, n3 = n * n * n;
    size_t nL = (size_t)E * n3;
#pragma omp parallel
    {
        double *ur = malloc(sizeof(double) * n3 * 6);
        double *us = ur + n3, *ut = us + n3, *vr = ut + n3, *vs = vr + n3, *vt = vs + n3;
#pragma omp for schedule(static)
        for (long e = 0; e < E; ++e) {
            size_t o = (size_t)e * n3;
            ref_grad(n, D, u + o, ur, us, ut);
            for (int p = 0; p < n3; ++p) {
                size_t q = o + p;
                double g11 = G[0 * nL + q], g22 = G[1 * nL + q], g33 = G[2 * nL + q];
                double g12 = G[3 * nL + q], g13 = G[4 * nL + q], g23 = G[5 * nL + q];
                vr[p] = h1 * (g11 * ur[p] + g12 * us[p] + g13 * ut[p]);
                vs[p] = h1 * (g12 * ur[p] + g22 * us[p] + g23 * ut[p]);
                vt[p] = h1 * (g13 * ur[p] + g23 * us[p] + g33 * ut[p]);
                w[q] = h2 * B[q] * u[q];
            }
            ref_grad_T(n, D, vr, vs, vt, w + o);
        }
        free(ur);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gather-scatter / direct-stiffness sum (Sec. 2: "gather/scatter")          */
/* ------------------------------------------------------------------------ */

/* Local copies of the unique index g along one direction of nel elements:
 * (element index, local index) pairs, in increasing element order. */
static int copies_1d(int g, int N, int nel, int periodic, int ce[2], int ci[2])
{
    int m = 0;
    if (g % N != 0) { ce[0] = g / N; ci[0] = g % N; return 1; }
    int e = g / N;
    if (periodic) {
        int eprev = (e - 1 + nel) % nel;
        /* order by element index */
        if (eprev < e) { ce[m] = eprev; ci[m++] = N; ce[m] = e; ci[m++] = 0; }
        else { ce[m] = e; ci[m++] = 0; ce[m] = eprev; ci[m++] = N; }
        return m;
    }
    if (e >= 1) { ce[m] = e - 1; ci[m++] = N; }
    if (e < nel) { ce[m] = e; ci[m++] = 0; }
    return m;
}

/* For each unique node, s = sum of all its local copies (summed in order of
 * element index then local node), then s is written back to every copy
 * (Q Q^T u).  Periodic directions identify g and g + nel*N. */
int orc_dssum(int N, int nelx, int nely, int nelz, const int *periodic, double *u)
{
    if (N < 1 || N > ORC_NMAX) return ORC_ERR_ARG;
    int n = N + 1, n3 = n * n * n;
    long ngx = (long)nelx * N + (periodic[0] ? 0 : 1);
    long ngy = (long)nely * N + (periodic[1] ? 0 : 1);
    long ngz = (long)nelz * N + (periodic[2] ? 0 : 1);
#pragma omp parallel for schedule(static)
    for (long gz = 0; gz < ngz; ++gz)
        for (long gy = 0; gy < ngy; ++gy)
            for (long gx = 0; gx < ngx; ++gx) {
                int ex[2], ix[2], ey[2], iy[2], ez[2], iz[2];
                int mx = copies_1d((int)gx, N, nelx, periodic[0], ex, ix);
                int my = copies_1d((int)gy, N, nely, periodic[1], ey, iy);
                int mz = copies_1d((int)gz, N, nelz, periodic[2], ez, iz);
                if (mx * my * mz == 1) continue;
                /* collect (element, local node) pairs and sort lexicographically */
                size_t idx[8]; long key[8]; int m = 0;
                for (int c = 0; c < mz; ++c)
                    for (int b = 0; b < my; ++b)
                        for (int a = 0; a < mx; ++a) {
                            long e = ex[a] + (long)nelx * (ey[b] + (long)nely * ez[c]);
                            int l = (iz[c] * n + iy[b]) * n + ix[a];
                            key[m] = e * n3 + l;
                            idx[m++] = (size_t)e * n3 + l;
                        }
                for (int s = 1; s < m; ++s)
                    for (int t = s; t > 0 && key[t] < key[t - 1]; --t) {
                        long kk = key[t]; key[t] = key[t - 1]; key[t - 1] = kk;
                        size_t ii = idx[t]; idx[t] = idx[t - 1]; idx[t - 1] = ii;
                    }
                double s = 0;
                for (int t = 0; t < m; ++t) s += u[idx[t]];
                for (int t = 0; t < m; ++t) u[idx[t]] = s;
            }
    return ORC_OK;
}

/* Multiplicity of every local node: dssum of ones. */
int orc_mult(int N, int nelx, int nely, int nelz, const int *periodic, double *mult)
{
    size_t nL = (size_t)nelx * nely * nelz * (N + 1) * (N + 1) * (N + 1);
    for (size_t p = 0; p < nL; ++p) mult[p] = 1.0;
    return orc_dssum(N, nelx, nely, nelz, periodic, mult);
}

/* ------------------------------------------------------------------------ */
/* Reductions (glsc3: Sec. 2, Fig. 4 velocity hotspot kernel)               */
/* ------------------------------------------------------------------------ */

/* sum_p a_p b_p c_p with c = 1/mult, i.e. the assembled inner product;
 * per-element partial sums added in element order. */
double orc_glsc3(long E, int n3, const double *a, const double *b, const double *c)
{
    double *part = malloc(sizeof(double) * (E > 0 ? E : 1));
#pragma omp parallel for schedule(static)
    for (long e = 0; e < E; ++e) {
        double s = 0;
        for (int p = 0; p < n3; ++p) {
            size_t q = (size_t)e * n3 + p;
            s += a[q] * b[q] * c[q];
        }
        part[e] = s;
    }
    double s = 0;
    for (long e = 0; e < E; ++e) s += part[e];
    free(part);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Jacobi diagonal (Sec. 1.1: CG with the Jacobi preconditioner)             */
/* ------------------------------------------------------------------------ */

/* minv = 1 / dssum(diag(A_local)), with the exact diagonal of the local
 * operator, cross terms included:
 *  diag = h1 [ sum_l D_li^2 G11(l,j,k) + sum_l D_lj^2 G22(i,l,k)
 *            + sum_l D_lk^2 G33(i,j,l) + 2 D_ii D_jj G12 + 2 D_ii D_kk G13
 *            + 2 D_jj D_kk G23 ] + h2 B. */
int orc_jacobi(int N, int nelx, int nely, int nelz, const int *periodic, const double *D,
               const double *G, const double *B, double h1, double h2, double *minv)
{
    int n = N + 1, n3 = n * n * n;
    long E = (long)nelx * nely * nelz;
    size_t nL = (size_t)E * n3;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < E; ++e)
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    size_t o = (size_t)e * n3, q = o + (size_t)(k * n + j) * n + i;
                    double s = 0;
                    for (int l = 0; l < n; ++l) {
                        s += D[l * n + i] * D[l * n + i] * G[0 * nL + o + (k * n + j) * n + l];
                        s += D[l * n + j] * D[l * n + j] * G[1 * nL + o + (k * n + l) * n + i];
                        s += D[l * n + k] * D[l * n + k] * G[2 * nL + o + (l * n + j) * n + i];
                    }
                    s += 2 * D[i * n + i] * D[j * n + j] * G[3 * nL + q];
                    s += 2 * D[i * n + i] * D[k * n + k] * G[4 * nL + q];
                    s += 2 * D[j * n + j] * D[k * n + k] * G[5 * nL + q];
                    minv[q] = h1 * s + h2 * B[q];
                }
    orc_dssum(N, nelx, nely, nelz, periodic, minv);
    for (size_t q = 0; q < nL; ++q) minv[q] = 1.0 / minv[q];
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Jacobi preconditioned CG (Sec. 1.1, Sec. 3: velocity CG+Jacobi)          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, nelx, nely, nelz, periodic[3];
    const double *D, *G, *B;
} orc_op;

/* y = dssum(A x) */
static void apply_A(const orc_op *op, double h1, double h2, const double *x, double *y)
{
    long E = (long)op->nelx * op->nely * op->nelz;
    orc_ax(op->N, E, op->D, op->G, op->B, h1, h2, x, y);
    orc_dssum(op->N, op->nelx, op->nely, op->nelz, op->periodic, y);
}

/* Jacobi-PCG on dssum(A) x = b.  The inner product is
 * <a,b> = sum_local a b / mult.  Stopping test ||r|| <= tol * ||b|| (relative)
 * or ||r|| <= tol (abs_tol != 0).  With h2 == 0 the operator has the
 * constants in its null space: b loses its mean (b -= <b,1>/<1,1>) before the
 * iteration and x loses its B-weighted mean after it.  Breakdown when
 * <p,Ap> <= 0 or is not finite.  x holds x0 on entry, the last iterate on
 * exit.  out[0] = iterations, out[1] = final ||r||, out[2] = ||b||. */
int orc_pcg(int N, int nelx, int nely, int nelz, const int *periodic, const double *D,
            const double *G, const double *B, double h1, double h2, const double *b_in,
            double *x, double tol, int abs_tol, int maxit, double *out)
{
    int n = N + 1, n3 = n * n * n;
    long E = (long)nelx * nely * nelz;
    size_t nL = (size_t)E * n3;
    orc_op op = {N, nelx, nely, nelz, {periodic[0], periodic[1], periodic[2]}, D, G, B};
    double *mult = malloc(sizeof(double) * nL * 7);
    double *imult = mult + nL, *minv = imult + nL, *r = minv + nL, *z = r + nL, *p = z + nL,
           *w = p + nL;
    orc_mult(N, nelx, nely, nelz, periodic, mult);
    for (size_t q = 0; q < nL; ++q) imult[q] = 1.0 / mult[q];
    orc_jacobi(N, nelx, nely, nelz, periodic, D, G, B, h1, h2, minv);
    int singular = (h2 == 0.0);
    double *b = malloc(sizeof(double) * nL);
    memcpy(b, b_in, sizeof(double) * nL);
    if (singular) {
        double *one = malloc(sizeof(double) * nL);
        for (size_t q = 0; q < nL; ++q) one[q] = 1.0;
        double mb = orc_glsc3(E, n3, b, one, imult) / orc_glsc3(E, n3, one, one, imult);
        for (size_t q = 0; q < nL; ++q) b[q] -= mb;
        free(one);
    }
    double bnorm = sqrt(orc_glsc3(E, n3, b, b, imult));
    apply_A(&op, h1, h2, x, w);
    for (size_t q = 0; q < nL; ++q) r[q] = b[q] - w[q];
    double rnorm = sqrt(orc_glsc3(E, n3, r, r, imult));
    double target = abs_tol ? tol : tol * bnorm;
    int status = ORC_OK, it = 0;
    if (!isfinite(rnorm) || !isfinite(bnorm)) status = ORC_ERR_BREAKDOWN;
    else if (rnorm > target) {
        for (size_t q = 0; q < nL; ++q) { z[q] = minv[q] * r[q]; p[q] = z[q]; }
        double rz = orc_glsc3(E, n3, r, z, imult);
        status = ORC_ERR_NOT_CONVERGED;
        for (it = 1; it <= maxit; ++it) {
            apply_A(&op, h1, h2, p, w);
            double pw = orc_glsc3(E, n3, p, w, imult);
            if (!(pw > 0) || !isfinite(pw)) { status = ORC_ERR_BREAKDOWN; break; }
            double alpha = rz / pw;
            for (size_t q = 0; q < nL; ++q) { x[q] += alpha * p[q]; r[q] -= alpha * w[q]; }
            rnorm = sqrt(orc_glsc3(E, n3, r, r, imult));
            if (!isfinite(rnorm)) { status = ORC_ERR_BREAKDOWN; break; }
            if (rnorm <= target) { status = ORC_OK; break; }
            for (size_t q = 0; q < nL; ++q) z[q] = minv[q] * r[q];
            double rz1 = orc_glsc3(E, n3, r, z, imult);
            double beta = rz1 / rz;
            rz = rz1;
            for (size_t q = 0; q < nL; ++q) p[q] = z[q] + beta * p[q];
        }
        if (it > maxit) it = maxit;
    }
    if (singular) {
        double sbx = 0, sb = 0;
        double *part = malloc(sizeof(double) * 2 * E);
#pragma omp parallel for schedule(static)
        for (long e = 0; e < E; ++e) {
            double a = 0, c = 0;
            for (int q = 0; q < n3; ++q) { a += B[(size_t)e * n3 + q] * x[(size_t)e * n3 + q]; c += B[(size_t)e * n3 + q]; }
            part[2 * e] = a; part[2 * e + 1] = c;
        }
        for (long e = 0; e < E; ++e) { sbx += part[2 * e]; sb += part[2 * e + 1]; }
        free(part);
        double m = sbx / sb;
        for (size_t q = 0; q < nL; ++q) x[q] -= m;
    }
    out[0] = it; out[1] = rnorm; out[2] = bnorm;
    free(b);
    free(mult);
    return status;
}

/* FP64 residual of a given x: r = b' - dssum(A x) with b' = b minus its mean
 * when h2 == 0.  out[0] = ||r||, out[1] = ||b'|| (assembled norms); r may be
 * NULL. */
int orc_residual(int N, int nelx, int nely, int nelz, const int *periodic, const double *D,
                 const double *G, const double *B, double h1, double h2, const double *b_in,
                 const double *x, double *r_out, double *out)
{
    int n = N + 1, n3 = n * n * n;
    long E = (long)nelx * nely * nelz;
    size_t nL = (size_t)E * n3;
    orc_op op = {N, nelx, nely, nelz, {periodic[0], periodic[1], periodic[2]}, D, G, B};
    double *imult = malloc(sizeof(double) * nL * 3), *b = imult + nL, *w = b + nL;
    orc_mult(N, nelx, nely, nelz, periodic, imult);
    for (size_t q = 0; q < nL; ++q) imult[q] = 1.0 / imult[q];
    memcpy(b, b_in, sizeof(double) * nL);
    if (h2 == 0.0) {
        double sb = 0, s1 = 0;
        double *one = malloc(sizeof(double) * nL);
        for (size_t q = 0; q < nL; ++q) one[q] = 1.0;
        sb = orc_glsc3(E, n3, b, one, imult);
        s1 = orc_glsc3(E, n3, one, one, imult);
        for (size_t q = 0; q < nL; ++q) b[q] -= sb / s1;
        free(one);
    }
    apply_A(&op, h1, h2, x, w);
    for (size_t q = 0; q < nL; ++q) w[q] = b[q] - w[q];
    out[0] = sqrt(orc_glsc3(E, n3, w, w, imult));
    out[1] = sqrt(orc_glsc3(E, n3, b, b, imult));
    if (r_out) memcpy(r_out, w, sizeof(double) * nL);
    free(imult);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dealiased convective term (adv_dealias: Sec. 1.1 Fig. 3, Table 2 B-5)     */
/* ------------------------------------------------------------------------ */

/* v = (A x A x A) u for one element, A is m x n (row-major), u is n^3,
 * v is m^3, applied one direction at a time. */
static void tensor3(int m, int n, const double *A, const double *u, double *v, double *t1, double *t2)
{
    /* along i: t1[k][j][q] */
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int q = 0; q < m; ++q) {
                double s = 0;
                for (int l = 0; l < n; ++l) s += A[q * n + l] * u[(k * n + j) * n + l];
                t1[(k * n + j) * m + q] = s;
            }
    /* along j: t2[k][q2][q] */
    for (int k = 0; k < n; ++k)
        for (int q2 = 0; q2 < m; ++q2)
            for (int q = 0; q < m; ++q) {
                double s = 0;
                for (int l = 0; l < n; ++l) s += A[q2 * n + l] * t1[(k * n + l) * m + q];
                t2[(k * m + q2) * m + q] = s;
            }
    /* along k */
    for (int q3 = 0; q3 < m; ++q3)
        for (int q2 = 0; q2 < m; ++q2)
            for (int q = 0; q < m; ++q) {
                double s = 0;
                for (int l = 0; l < n; ++l) s += A[q3 * n + l] * t2[(l * m + q2) * m + q];
                v[(q3 * m + q2) * m + q] = s;
            }
}

/* out = (A^T x A^T x A^T) f for one element, A is m x n, f is m^3, out n^3. */
static void tensor3_T(int m, int n, const double *A, const double *f, double *out, double *t1, double *t2)
{
    for (int q3 = 0; q3 < m; ++q3)
        for (int q2 = 0; q2 < m; ++q2)
            for (int i = 0; i < n; ++i) {
                double s = 0;
                for (int q = 0; q < m; ++q) s += A[q * n + i] * f[(q3 * m + q2) * m + q];
                t1[(q3 * m + q2) * n + i] = s;
            }
    for (int q3 = 0; q3 < m; ++q3)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double s = 0;
                for (int q = 0; q < m; ++q) s += A[q * n + j] * t1[(q3 * m + q) * n + i];
                t2[(q3 * n + j) * n + i] = s;
            }
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double s = 0;
                for (int q = 0; q < m; ++q) s += A[q * n + k] * t2[(q * n + j) * n + i];
                out[(k * n + j) * n + i] = s;
            }
}

/* Number of Gauss-Legendre points per direction of the dealiasing grid:
 * M = ceil(3(N+1)/2) (3/2 rule). */
int orc_dealias_m(int N) { return (3 * (N + 1) + 1) / 2; }

/* Weak dealiased convective term C_c = int phi (u . grad) u_c on each element:
 *  1. physical gradient on GLL: du_c/dx_d = sum_a (dr_a/dx_d) (D_a u_c),
 *  2. interpolate u_d and du_c/dx_d to the M^3 GL points (J_qj = l_j(eta_q)),
 *  3. f_c = W_q |J(eta_q)| sum_d u_d (du_c/dx_d)   with |J| from the trilinear map,
 *  4. C_c = (J^T x J^T x J^T) f_c.
 * Local (not assembled).  u[c] and C[c] are E-vectors (c = 0..2). */
int orc_convect(int N, int nelx, int nely, int nelz, const double *vert, const double *jinv,
                const double *u0, const double *u1, const double *u2,
                double *C0, double *C1, double *C2)
{
    int n = N + 1, n3 = n * n * n, M = orc_dealias_m(N), m3 = M * M * M;
    long E = (long)nelx * nely * nelz;
    size_t nL = (size_t)E * n3;
    double xi[ORC_NMAX + 1], w[ORC_NMAX + 1], D[(ORC_NMAX + 1) * (ORC_NMAX + 1)];
    double eta[64], wg[64];
    orc_gll(N, xi, w);
    orc_deriv(N, xi, D);
    orc_gl(M, eta, wg);
    double *J = malloc(sizeof(double) * M * n);
    orc_interp(N, xi, M, eta, J);
    const double *u[3] = {u0, u1, u2};
    double *C[3] = {C0, C1, C2};
#pragma omp parallel
    {
        double *buf = malloc(sizeof(double) * (size_t)(n3 * 3 + m3 * 3 + m3 * 9 + m3 * 3 + 2 * m3 + m3 + n3));
        double *ur = buf, *us = ur + n3, *ut = us + n3;
        double *fu = ut + n3;          /* 3 * m3: interpolated velocity */
        double *fg = fu + 3 * m3;      /* 9 * m3: interpolated gradient [c*3+d] */
        double *fdet = fg + 9 * m3;    /* m3 */
        double *t1 = fdet + m3, *t2 = t1 + m3, *f = t2 + m3, *g = f + m3;  /* g: n3 */
        /* fdet etc. only m3 each; trailing space reserved */
#pragma omp for schedule(static)
        for (long e = 0; e < E; ++e) {
            size_t o = (size_t)e * n3;
            double X[8][3];
            elem_vertices(nelx, nely, (int)e, vert, X);
            for (int d = 0; d < 3; ++d) tensor3(M, n, J, u[d] + o, fu + d * m3, t1, t2);
            for (int c = 0; c < 3; ++c) {
                ref_grad(n, D, u[c] + o, ur, us, ut);
                for (int d = 0; d < 3; ++d) {
                    for (int p = 0; p < n3; ++p) {
                        size_t q = o + p;
                        g[p] = jinv[(0 * 3 + d) * nL + q] * ur[p] + jinv[(1 * 3 + d) * nL + q] * us[p] +
                               jinv[(2 * 3 + d) * nL + q] * ut[p];
                    }
                    tensor3(M, n, J, g, fg + (c * 3 + d) * m3, t1, t2);
                }
            }
            for (int q3 = 0; q3 < M; ++q3)
                for (int q2 = 0; q2 < M; ++q2)
                    for (int q1 = 0; q1 < M; ++q1) {
                        double x[3], jac[3][3], inv[3][3];
                        trilinear(X, eta[q1], eta[q2], eta[q3], x, jac);
                        fdet[(q3 * M + q2) * M + q1] = wg[q1] * wg[q2] * wg[q3] * inv3(jac, inv);
                    }
            for (int c = 0; c < 3; ++c) {
                for (int q = 0; q < m3; ++q) {
                    double s = 0;
                    for (int d = 0; d < 3; ++d) s += fu[d * m3 + q] * fg[(c * 3 + d) * m3 + q];
                    f[q] = fdet[q] * s;
                }
                tensor3_T(M, n, J, f, C[c] + o, t1, t2);
            }
        }
        free(buf);
    }
    free(J);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* TGV diagnostics (Sec. 3; Sec. 4.2)                                        */
/* ------------------------------------------------------------------------ */

/* out[0] = KE = 1/(2V) sum_local B |u|^2,
 * out[1] = enstrophy = 1/(2V) sum_local B |curl u|^2 (element-local curl). */
int orc_diag(int N, long E, const double *D, const double *jinv, const double *B, double V,
             const double *u0, const double *u1, const double *u2, double *out)
{
    int n = N + 1, n3 = n * n * n;
    size_t nL = (size_t)E * n3;
    const double *u[3] = {u0, u1, u2};
    double *part = malloc(sizeof(double) * 2 * (E > 0 ? E : 1));
#pragma omp parallel
    {
        double *gr = malloc(sizeof(double) * n3 * 12);
#pragma omp for schedule(static)
        for (long e = 0; e < E; ++e) {
            size_t o = (size_t)e * n3;
            for (int c = 0; c < 3; ++c) ref_grad(n, D, u[c] + o, gr + (3 * c) * n3, gr + (3 * c + 1) * n3, gr + (3 * c + 2) * n3);
            double ke = 0, en = 0;
            for (int p = 0; p < n3; ++p) {
                size_t q = o + p;
                double du[3][3]; /* du[c][d] = du_c/dx_d */
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) {
                        double s = 0;
                        for (int a = 0; a < 3; ++a) s += jinv[(a * 3 + d) * nL + q] * gr[(3 * c + a) * n3 + p];
                        du[c][d] = s;
                    }
                double wx = du[2][1] - du[1][2], wy = du[0][2] - du[2][0], wz = du[1][0] - du[0][1];
                ke += B[q] * (u0[q] * u0[q] + u1[q] * u1[q] + u2[q] * u2[q]);
                en += B[q] * (wx * wx + wy * wy + wz * wz);
            }
            part[2 * e] = ke; part[2 * e + 1] = en;
        }
        free(gr);
    }
    double ke = 0, en = 0;
    for (long e = 0; e < E; ++e) { ke += part[2 * e]; en += part[2 * e + 1]; }
    free(part);
    out[0] = ke / (2 * V);
    out[1] = en / (2 * V);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* BDF3/EXT3 P_N-P_N step (Sec. 2, Fig. 3; Sec. 3)                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, nelx, nely, nelz, periodic[3];
    long E;
    size_t nL;
    double nu, dt, V, t;
    double hist_dt[2];              /* sizes of the last two steps taken (most recent first) */
    double cfl_target, dt_max, cfl; /* adaptive step (cfl_target > 0); CFL of the last step */
    double tol_v, tol_p;
    int abs_tol, maxit;
    int step;                       /* steps taken so far */
    int store32;                    /* stored state kept as FP32 values (rp = fp32, Table 2 group B) */
    double *vert, *D, *jinv, *G, *B, *Bsum;
    double *u[3][3];                /* u[h][c]: h = 0 -> u^n, 1 -> u^{n-1}, 2 -> u^{n-2} */
    double *C[3][3];                /* C[h][c]: convective term at the same levels */
    double *p;
    double *work;                   /* 4 * nL */
} orc_tgv;

/* BDF / EXT coefficients of order q for variable steps (Sec. 3: fixed third
 * order; the adaptive CFL step of Sec. 3 makes the steps unequal).  dts[0] is
 * the step being taken (t^n -> t^{n+1}), dts[1] and dts[2] the two before it.
 * With tau_0 = t^{n+1}, tau_j = t^{n+1-j} (j = 1..q):
 *   BDF: u'(tau_0) ~ sum_{j=0..q} l_j'(tau_0) u(tau_j) for the Lagrange basis
 *        l_j of tau_0..tau_q, written (b0 u^{n+1} - sum_j b_j u^{n+1-j}) / dts[0]:
 *        b0 = dts[0] l_0'(tau_0), b_j = -dts[0] l_j'(tau_0);
 *   EXT: u(tau_0) ~ sum_{j=1..q} a_j u(tau_j), a_j = prod_{k=1..q, k!=j}
 *        (tau_0 - tau_k) / (tau_j - tau_k).
 * Equal steps give the textbook values (11/6; 3, -3/2, 1/3; 3, -3, 1). */
void orc_bdf_ext_var(int q, const double *dts, double *b0, double *b, double *a)
{
    double tau[4];
    tau[0] = 0.0;
    for (int j = 1; j <= 3; ++j) tau[j] = tau[j - 1] - (j <= q ? dts[j - 1] : 1.0);
    b[0] = b[1] = b[2] = a[0] = a[1] = a[2] = 0;
    /* l_j'(tau_0) = sum_{m != j} 1/(tau_j - tau_m) prod_{k != j, m} (tau_0 - tau_k)/(tau_j - tau_k) */
    for (int j = 0; j <= q; ++j) {
        double d = 0.0;
        for (int m = 0; m <= q; ++m) {
            if (m == j) continue;
            double term = 1.0 / (tau[j] - tau[m]);
            for (int k = 0; k <= q; ++k)
                if (k != j && k != m) term *= (tau[0] - tau[k]) / (tau[j] - tau[k]);
            d += term;
        }
        if (j == 0) *b0 = dts[0] * d;
        else b[j - 1] = -dts[0] * d;
    }
    for (int j = 1; j <= q; ++j) {
        double l = 1.0;
        for (int k = 1; k <= q; ++k)
            if (k != j) l *= (tau[0] - tau[k]) / (tau[j] - tau[k]);
        a[j - 1] = l;
    }
}

static void bdf_ext(int q, const double dts[3], double *b0, double b[3], double a[3])
{
    orc_bdf_ext_var(q, dts, b0, b, a);
}

/* CFL number of a velocity field for a step dt (reading of Sec. 3's CFL 0.4):
 * dt * max over local nodes of sum_a |U_a| / dxi_a, with U_a = sum_c
 * (dr_a/dx_c) u_c the reference-space velocity and dxi_a the GLL spacing at
 * the node's index in direction a (the smaller of its two neighbour gaps). */
double orc_cfl(int N, long E, const double *jinv, const double *u0, const double *u1,
               const double *u2, double dt)
{
    int n = N + 1, n3 = n * n * n;
    size_t nL = (size_t)E * n3;
    double xi[ORC_NMAX + 1], w[ORC_NMAX + 1], gap[ORC_NMAX + 1];
    orc_gll(N, xi, w);
    for (int i = 0; i <= N; ++i) {
        double gl = i > 0 ? xi[i] - xi[i - 1] : 1e300, gr = i < N ? xi[i + 1] - xi[i] : 1e300;
        gap[i] = gl < gr ? gl : gr;
    }
    const double *u[3] = {u0, u1, u2};
    double m = 0.0;
#pragma omp parallel for reduction(max : m) schedule(static)
    for (long e = 0; e < E; ++e)
        for (int p = 0; p < n3; ++p) {
            size_t q = (size_t)e * n3 + p;
            int idx[3] = {p % n, (p / n) % n, p / (n * n)};
            double c = 0.0;
            for (int a = 0; a < 3; ++a) {
                double U = 0.0;
                for (int cc = 0; cc < 3; ++cc) U += jinv[(a * 3 + cc) * nL + q] * u[cc][q];
                c += fabs(U) / gap[idx[a]];
            }
            if (c > m) m = c;
        }
    return dt * m;
}

void *orc_tgv_create(int N, int nelx, int nely, int nelz, const double *vert, const double *L,
                     double nu, double dt, double tol_v, double tol_p, int abs_tol, int maxit)
{
    if (N < 1 || N > ORC_NMAX) return NULL;
    orc_tgv *s = calloc(1, sizeof(orc_tgv));
    int n = N + 1;
    s->N = N; s->nelx = nelx; s->nely = nely; s->nelz = nelz;
    s->periodic[0] = s->periodic[1] = s->periodic[2] = 1;
    s->E = (long)nelx * nely * nelz;
    s->nL = (size_t)s->E * n * n * n;
    s->nu = nu; s->dt = dt; s->V = L[0] * L[1] * L[2];
    s->tol_v = tol_v; s->tol_p = tol_p; s->abs_tol = abs_tol; s->maxit = maxit;
    size_t nv = (size_t)(nelx + 1) * (nely + 1) * (nelz + 1) * 3;
    s->vert = malloc(sizeof(double) * nv);
    memcpy(s->vert, vert, sizeof(double) * nv);
    double xi[ORC_NMAX + 1], w[ORC_NMAX + 1];
    s->D = malloc(sizeof(double) * n * n);
    orc_gll(N, xi, w);
    orc_deriv(N, xi, s->D);
    size_t nL = s->nL;
    s->jinv = malloc(sizeof(double) * 9 * nL);
    s->G = malloc(sizeof(double) * 6 * nL);
    s->B = malloc(sizeof(double) * nL);
    s->Bsum = malloc(sizeof(double) * nL);
    if (orc_geom(N, nelx, nely, nelz, vert, NULL, s->jinv, s->G, s->B) != ORC_OK) {
        free(s->vert); free(s->D); free(s->jinv); free(s->G); free(s->B); free(s->Bsum); free(s);
        return NULL;
    }
    memcpy(s->Bsum, s->B, sizeof(double) * nL);
    orc_dssum(N, nelx, nely, nelz, s->periodic, s->Bsum);
    for (int h = 0; h < 3; ++h)
        for (int c = 0; c < 3; ++c) {
            s->u[h][c] = calloc(nL, sizeof(double));
            s->C[h][c] = calloc(nL, sizeof(double));
        }
    s->p = calloc(nL, sizeof(double));
    s->work = calloc(4 * nL, sizeof(double));
    return s;
}

void orc_tgv_destroy(void *h)
{
    orc_tgv *s = h;
    if (!s) return;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) { free(s->u[a][c]); free(s->C[a][c]); }
    free(s->p); free(s->work); free(s->vert); free(s->D); free(s->jinv); free(s->G); free(s->B);
    free(s->Bsum); free(s);
}

/* Storage precision of the stepper's state (Sec. 4: the global precision rp
 * is the storage format).  store32 != 0: the convective term, the pressure and
 * the new velocity are rounded to FP32 values where each step stores them,
 * and so is the state given to orc_tgv_set after this call (with rp = fp32
 * the whole state is FP32 from the start); the arithmetic stays FP64. */
int orc_tgv_set_storage(void *hnd, int store32)
{
    orc_tgv *s = hnd;
    s->store32 = store32 != 0;
    return ORC_OK;
}

static void round_to_float(double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i) a[i] = (double)(float)a[i];
}

/* Set u^{n-h} (h = 0,1,2) and, for h == 0, p^n; the convective history at
 * level h is evaluated from the given field.  'step' sets the number of
 * steps already taken (it selects the startup BDF/EXT order). */
int orc_tgv_set(void *hnd, int h, const double *u0, const double *u1, const double *u2,
                const double *p, int step, double t)
{
    orc_tgv *s = hnd;
    if (h < 0 || h > 2) return ORC_ERR_ARG;
    memcpy(s->u[h][0], u0, sizeof(double) * s->nL);
    memcpy(s->u[h][1], u1, sizeof(double) * s->nL);
    memcpy(s->u[h][2], u2, sizeof(double) * s->nL);
    if (s->store32)
        for (int c = 0; c < 3; ++c) round_to_float(s->u[h][c], s->nL);
    orc_convect(s->N, s->nelx, s->nely, s->nelz, s->vert, s->jinv, s->u[h][0], s->u[h][1],
                s->u[h][2], s->C[h][0], s->C[h][1], s->C[h][2]);
    if (s->store32)
        for (int c = 0; c < 3; ++c) round_to_float(s->C[h][c], s->nL);
    if (h == 0) {
        if (p) memcpy(s->p, p, sizeof(double) * s->nL);
        if (p && s->store32) round_to_float(s->p, s->nL);
        s->step = step;
        s->t = t;
        s->hist_dt[0] = s->hist_dt[1] = s->dt;  /* earlier levels: steps of the current size */
    }
    return ORC_OK;
}

/* Adaptive step (cfl_target > 0; 0 keeps dt fixed) and the step of the next
 * step (dt > 0; 0 keeps it). */
int orc_tgv_set_dt(void *hnd, double dt, double cfl_target, double dt_max)
{
    orc_tgv *s = hnd;
    if (dt > 0) s->dt = dt;
    s->cfl_target = cfl_target > 0 ? cfl_target : 0.0;
    s->dt_max = dt_max > 0 ? dt_max : 0.0;
    return ORC_OK;
}

int orc_tgv_get(void *hnd, double *u0, double *u1, double *u2, double *p)
{
    orc_tgv *s = hnd;
    memcpy(u0, s->u[0][0], sizeof(double) * s->nL);
    memcpy(u1, s->u[0][1], sizeof(double) * s->nL);
    memcpy(u2, s->u[0][2], sizeof(double) * s->nL);
    if (p) memcpy(p, s->p, sizeof(double) * s->nL);
    return ORC_OK;
}

/* One or more P_N-P_N steps.  Per step (order q = min(step+1, 3)):
 *  1. C^n_c = dealiased convective term of u^n (the history levels C^{n-1},
 *     C^{n-2} are kept from earlier steps),
 *  2. F_c = -sum_j a_j C^{n+1-j}_c                       (EXT, weak, local)
 *  3. g_c = Bsum^{-1} dssum(F_c) + sum_j (b_j/dt) u^{n+1-j}_c   (strong)
 *  4. A p^{n+1} = dssum( sum_c Dt_c^T g_c ) with Dt_c^T the weak divergence,
 *     (Dt_c^T g)_i = sum_q B_q (d phi_i/dx_c)(q) g(q); PCG from p^n,
 *     h1 = 1, h2 = 0 (singular: mean removal)
 *  5. (nu A + (b0/dt) B) u^{n+1}_c = dssum( F_c + B sum_j (b_j/dt) u^{n+1-j}_c
 *                                           - B dp/dx_c ),  PCG from sum_j a_j u^{n+1-j}_c,
 *  6. shift histories; diagnostics KE, enstrophy at t^{n+1}.
 * diag[s*10 + ...] = {t, KE, enstrophy, it_p, it_u, it_v, it_w, status, dt of the
 * step, CFL of the new velocity for that dt}. */
int orc_tgv_step(void *hnd, int nsteps, double *diag)
{
    orc_tgv *s = hnd;
    int N = s->N, n = N + 1, n3 = n * n * n;
    size_t nL = s->nL;
    long E = s->E;
    double *F[3], *g[3];
    double *tmp = s->work + 3 * nL;
    int rc_all = ORC_OK;
    for (int c = 0; c < 3; ++c) F[c] = s->work + c * nL;
    for (int c = 0; c < 3; ++c) g[c] = malloc(sizeof(double) * nL);
    double *bp = malloc(sizeof(double) * nL);
    double *rhs = malloc(sizeof(double) * nL);
    double *gr = malloc(sizeof(double) * 3 * nL);
    for (int st = 0; st < nsteps; ++st) {
        int q = s->step + 1 < 3 ? s->step + 1 : 3;
        double b0, b[3], a[3];
        double dt = s->dt;
        const double dts[3] = {dt, s->hist_dt[0], s->hist_dt[1]};
        bdf_ext(q, dts, &b0, b, a);
        /* 1. convective term at level n (C[0] holds it after the previous step's shift) */
        orc_convect(N, s->nelx, s->nely, s->nelz, s->vert, s->jinv, s->u[0][0], s->u[0][1],
                    s->u[0][2], s->C[0][0], s->C[0][1], s->C[0][2]);
        if (s->store32)
            for (int c = 0; c < 3; ++c) round_to_float(s->C[0][c], nL);
        /* 2-3. */
        for (int c = 0; c < 3; ++c) {
            for (size_t p = 0; p < nL; ++p)
                F[c][p] = -(a[0] * s->C[0][c][p] + a[1] * s->C[1][c][p] + a[2] * s->C[2][c][p]);
            memcpy(tmp, F[c], sizeof(double) * nL);
            orc_dssum(N, s->nelx, s->nely, s->nelz, s->periodic, tmp);
            for (size_t p = 0; p < nL; ++p)
                g[c][p] = tmp[p] / s->Bsum[p] +
                          (b[0] * s->u[0][c][p] + b[1] * s->u[1][c][p] + b[2] * s->u[2][c][p]) / dt;
        }
        /* 4. pressure RHS: sum_a D_a^T ( B sum_c (dr_a/dx_c) g_c ) */
#pragma omp parallel
        {
            double *h = malloc(sizeof(double) * 3 * n3);
#pragma omp for schedule(static)
            for (long e = 0; e < E; ++e) {
                size_t o = (size_t)e * n3;
                for (int pp = 0; pp < n3; ++pp) {
                    size_t qq = o + pp;
                    for (int aa = 0; aa < 3; ++aa) {
                        double v = 0;
                        for (int c = 0; c < 3; ++c) v += s->jinv[(aa * 3 + c) * nL + qq] * g[c][qq];
                        h[aa * n3 + pp] = s->B[qq] * v;
                    }
                    bp[qq] = 0;
                }
                ref_grad_T(n, s->D, h, h + n3, h + 2 * n3, bp + o);
            }
            free(h);
        }
        orc_dssum(N, s->nelx, s->nely, s->nelz, s->periodic, bp);
        double info[3];
        int rc = orc_pcg(N, s->nelx, s->nely, s->nelz, s->periodic, s->D, s->G, s->B, 1.0, 0.0, bp,
                         s->p, s->tol_p, s->abs_tol, s->maxit, info);
        int itp = (int)info[0];
        if (rc != ORC_OK) rc_all = rc;
        if (s->store32) round_to_float(s->p, nL);
        /* 5. pressure gradient (element-local) and velocity solves */
#pragma omp parallel
        {
            double *pr = malloc(sizeof(double) * 3 * n3);
#pragma omp for schedule(static)
            for (long e = 0; e < E; ++e) {
                size_t o = (size_t)e * n3;
                ref_grad(n, s->D, s->p + o, pr, pr + n3, pr + 2 * n3);
                for (int pp = 0; pp < n3; ++pp)
                    for (int c = 0; c < 3; ++c) {
                        double v = 0;
                        for (int aa = 0; aa < 3; ++aa) v += s->jinv[(aa * 3 + c) * nL + o + pp] * pr[aa * n3 + pp];
                        gr[c * nL + o + pp] = v;
                    }
            }
            free(pr);
        }
        int itu[3];
        for (int c = 0; c < 3; ++c) {
            for (size_t p = 0; p < nL; ++p)
                rhs[p] = F[c][p] +
                         s->B[p] * ((b[0] * s->u[0][c][p] + b[1] * s->u[1][c][p] + b[2] * s->u[2][c][p]) / dt -
                                    gr[c * nL + p]);
            orc_dssum(N, s->nelx, s->nely, s->nelz, s->periodic, rhs);
            /* new velocity goes into the oldest level, which is shifted out; the
             * solve starts from the extrapolated velocity sum_j a_j u^{n+1-j}
             * (the EXT weights of this step; this build's reading: the paper does
             * not state the initial guess) */
            for (size_t p = 0; p < nL; ++p)
                s->u[2][c][p] = a[0] * s->u[0][c][p] + a[1] * s->u[1][c][p] + a[2] * s->u[2][c][p];
            rc = orc_pcg(N, s->nelx, s->nely, s->nelz, s->periodic, s->D, s->G, s->B, s->nu, b0 / dt,
                         rhs, s->u[2][c], s->tol_v, s->abs_tol, s->maxit, info);
            itu[c] = (int)info[0];
            if (rc != ORC_OK) rc_all = rc;
        }
        /* 6. shift: level 2 holds u^{n+1}; rotate so that level 0 is u^{n+1} */
        for (int c = 0; c < 3; ++c) {
            double *un1 = s->u[2][c];
            s->u[2][c] = s->u[1][c];
            s->u[1][c] = s->u[0][c];
            s->u[0][c] = un1;
            double *cn = s->C[2][c];
            s->C[2][c] = s->C[1][c];
            s->C[1][c] = s->C[0][c];
            s->C[0][c] = cn; /* overwritten by the next step's convective evaluation */
            if (s->store32) round_to_float(s->u[0][c], nL);
        }
        s->step += 1;
        s->t += dt;
        s->hist_dt[1] = s->hist_dt[0];
        s->hist_dt[0] = dt;
        double d[2];
        orc_diag(N, E, s->D, s->jinv, s->B, s->V, s->u[0][0], s->u[0][1], s->u[0][2], d);
        /* CFL of the new velocity for the step just taken; the adaptive rule
         * (reading) scales the next step towards the target, by at most +10 %
         * and -50 % per step, capped by dt_max */
        s->cfl = orc_cfl(N, E, s->jinv, s->u[0][0], s->u[0][1], s->u[0][2], dt);
        if (s->cfl_target > 0 && s->cfl > 0) {
            double f = s->cfl_target / s->cfl;
            if (f > 1.1) f = 1.1;
            if (f < 0.5) f = 0.5;
            s->dt = dt * f;
            if (s->dt_max > 0 && s->dt > s->dt_max) s->dt = s->dt_max;
        }
        if (diag) {
            double *o = diag + 10 * st;
            o[0] = s->t; o[1] = d[0]; o[2] = d[1];
            o[3] = itp; o[4] = itu[0]; o[5] = itu[1]; o[6] = itu[2]; o[7] = rc_all;
            o[8] = dt; o[9] = s->cfl;
        }
    }
    for (int c = 0; c < 3; ++c) free(g[c]);
    free(bp); free(rhs); free(gr);
    return rc_all;
}

/* ------------------------------------------------------------------------ */
/* Analytic right-hand side: a finite Fourier series at given points         */
/* ------------------------------------------------------------------------ */

/* out[p] = sum_m cc[m] cos(k_m . x_p) + cs[m] sin(k_m . x_p), k_m integer with
 * |k| components <= kmax; e^{i k.x} built from tabulated integer powers of
 * e^{ix}, e^{iy}, e^{iz}.  (Input generation for the pressure-Poisson
 * workload: the divergence of a random smooth velocity field.) */
int orc_fourier(long nm, const long *K, const double *cc, const double *cs, long npts,
                const double *x, const double *y, const double *z, int kmax, double *out)
{
    if (kmax < 0 || kmax > 32) return ORC_ERR_ARG;
    int w = 2 * kmax + 1;
#pragma omp parallel
    {
        double *tab = malloc(sizeof(double) * 6 * w);
#pragma omp for schedule(static)
        for (long p = 0; p < npts; ++p) {
            const double c3[3] = {x[p], y[p], z[p]};
            for (int d = 0; d < 3; ++d) {
                double *re = tab + (2 * d) * w, *im = re + w;
                double cr = cos(c3[d]), ci = sin(c3[d]);
                re[kmax] = 1.0; im[kmax] = 0.0;
                for (int q = 1; q <= kmax; ++q) {
                    re[kmax + q] = re[kmax + q - 1] * cr - im[kmax + q - 1] * ci;
                    im[kmax + q] = re[kmax + q - 1] * ci + im[kmax + q - 1] * cr;
                    re[kmax - q] = re[kmax + q];
                    im[kmax - q] = -im[kmax + q];
                }
            }
            double s = 0.0;
            for (long m = 0; m < nm; ++m) {
                int a = (int)K[3 * m] + kmax, b = (int)K[3 * m + 1] + kmax, cidx = (int)K[3 * m + 2] + kmax;
                double ar = tab[a], ai = tab[w + a];
                double br = tab[2 * w + b], bi = tab[3 * w + b];
                double zr = tab[4 * w + cidx], zi = tab[5 * w + cidx];
                double tr = ar * br - ai * bi, ti = ar * bi + ai * br;
                double er = tr * zr - ti * zi, ei = tr * zi + ti * zr;
                s += cc[m] * er + cs[m] * ei;
            }
            out[p] = s;
        }
        free(tab);
    }
    return ORC_OK;
}
