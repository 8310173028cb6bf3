/*
 * sem_oracle_hsmg.c -- plain FP64 CPU oracle of the paper's pressure solver:
 * GMRES preconditioned by a three-level hybrid Schwarz multigrid (HSMG) whose
 * coarsest problem is solved by CG with the Jacobi preconditioner (Sec. 1 and
 * the solver settings of Sec. 3).
 *
 * THIS IS TEST INFRASTRUCTURE, under the same rules as sem_oracle.c (only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it; it shares nothing with the CUDA library).
 *
 * The paper names the method and its levels but prints none of its
 * definitions.  The ones below are the textbook constructions (overlapping
 * Schwarz smoothing with fast-diagonalisation local solves: Fischer,
 * "An overlapping Schwarz method for spectral element solution of the
 * incompressible Navier-Stokes equations", JCP 133, 1997; hybrid Schwarz
 * multigrid: Lottes & Fischer, J. Sci. Comput. 24, 2005; flexible GMRES:
 * Saad, SISC 14, 1993), with these readings:
 *  - levels: polynomial orders (N, N_mid, 1) on the same mesh, each level's
 *    operator the SEM operator of that order (its own geometric factors);
 *  - smoother: z = dssum(W sum_e R_e^T A~_e^{-1} R_e r), W = 1/multiplicity,
 *    A~_e the separable (box) approximation of the element's operator,
 *    extended at each face by the linear segment to the neighbour's first
 *    interior GLL node with a zero value there (one-node overlap), inverted
 *    by fast diagonalisation;
 *  - grid transfer: prolongation = tensor Lagrange interpolation from the
 *    coarser GLL points, restriction its transpose on unique nodes;
 *  - one V-cycle per application: smooth, restrict the residual, recurse,
 *    prolong and add; CG + Jacobi on the coarsest level to a relative
 *    tolerance;
 *  - GMRES is right-preconditioned and flexible (the preconditioner varies
 *    with the coarse solve), restarted after m steps, with modified
 *    Gram-Schmidt and Givens rotations, in the assembled inner product.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_NOT_CONVERGED -5
#define ORC_ERR_BREAKDOWN -6
#define ORC_NMAX 15

/* from sem_oracle.c */
int orc_gll(int N, double *xi, double *w);
int orc_deriv(int N, const double *xi, double *D);
int orc_interp(int N, const double *xi, int M, const double *x, double *J);
int orc_geom(int N, int nelx, int nely, int nelz, const double *vert, double *xyz, double *jinv,
             double *G, double *B);
int orc_ax(int N, long E, const double *D, const double *G, const double *B, double h1, double h2,
           const double *u, double *w);
int orc_dssum(int N, int nelx, int nely, int nelz, const int *periodic, double *u);
int orc_mult(int N, int nelx, int nely, int nelz, const int *periodic, double *mult);
double orc_glsc3(long E, int n3, const double *a, const double *b, const double *c);
int orc_pcg(int N, int nelx, int nely, int nelz, const int *periodic, const double *D,
            const double *G, const double *B, double h1, double h2, const double *b_in, double *x,
            double tol, int abs_tol, int maxit, double *out);

/* ------------------------------------------------------------------------ */
/* Symmetric eigenproblem (cyclic Jacobi rotations, Golub & Van Loan 8.5)    */
/* ------------------------------------------------------------------------ */

/* A (n x n, symmetric, row-major) = Q diag(lam) Q^T; A is destroyed; Q
 * column-major by eigenvector: Q[i*n + k] = i-th entry of eigenvector k. */
static void sym_eig(int n, double *A, double *lam, double *Q)
{
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) Q[i * n + k] = (i == k);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                tot += A[i * n + k] * A[i * n + k];
                if (i != k) off += A[i * n + k] * A[i * n + k];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                double c = 1 / sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < n; ++k) {  /* A <- A J (columns p, q) */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  /* A <- J^T A (rows p, q) */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  /* Q <- Q J */
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - s * qkq;
                    Q[k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

/* ------------------------------------------------------------------------ */
/* 1-D factors of the fast-diagonalisation local solve                       */
/* ------------------------------------------------------------------------ */

/* The extended 1-D operators of an element of length h whose neighbours have
 * lengths hl, hr (0 = no neighbour on that side):
 *   K = (2/h) Khat + diag(1/dl, 0, ..., 0, 1/dr),   Khat_ij = sum_q w_q D_qi D_qj,
 *   M = (h/2) diag(w) + diag(dl/2, 0, ..., 0, dr/2),
 * with dl = (xi_1 - xi_0) hl / 2 the distance to the left neighbour's first
 * interior GLL node (likewise dr): the linear segment to that node, whose far
 * end is held at zero, stiffens (and adds lumped mass to) the face node.
 * Output the generalised eigenpairs K S = M S diag(lam), S^T M S = I:
 * S[i*n + k] = entry i of eigenvector k.  Kout / Mout (may be NULL) receive
 * K and the diagonal of M. */
int orc_fdm_1d(int N, double h, double hl, double hr, double *S, double *lam, double *Kout,
               double *Mout)
{
    if (N < 1 || N > ORC_NMAX || !(h > 0)) return ORC_ERR_ARG;
    int n = N + 1;
    double xi[ORC_NMAX + 1], w[ORC_NMAX + 1], D[(ORC_NMAX + 1) * (ORC_NMAX + 1)];
    double K[(ORC_NMAX + 1) * (ORC_NMAX + 1)], M[ORC_NMAX + 1], C[(ORC_NMAX + 1) * (ORC_NMAX + 1)];
    double Q[(ORC_NMAX + 1) * (ORC_NMAX + 1)];
    orc_gll(N, xi, w);
    orc_deriv(N, xi, D);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0;
            for (int q = 0; q < n; ++q) s += w[q] * D[q * n + i] * D[q * n + j];
            K[i * n + j] = 2.0 / h * s;
        }
    for (int i = 0; i < n; ++i) M[i] = 0.5 * h * w[i];
    double gap = xi[1] - xi[0];
    if (hl > 0) {
        double d = 0.5 * gap * hl;
        K[0] += 1.0 / d;
        M[0] += 0.5 * d;
    }
    if (hr > 0) {
        double d = 0.5 * gap * hr;
        K[(n - 1) * n + n - 1] += 1.0 / d;
        M[n - 1] += 0.5 * d;
    }
    if (Kout) memcpy(Kout, K, sizeof(double) * n * n);
    if (Mout) memcpy(Mout, M, sizeof(double) * n);
    /* C = M^{-1/2} K M^{-1/2} = Q lam Q^T, S = M^{-1/2} Q */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) C[i * n + j] = K[i * n + j] / sqrt(M[i] * M[j]);
    sym_eig(n, C, lam, Q);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) S[i * n + k] = Q[i * n + k] / sqrt(M[i]);
    return ORC_OK;
}

/* z = A~^{-1} r on one element: A~ = h1 (Mz x My x Kx + Mz x Ky x Mx + Kz x My x Mx)
 * + h2 (Mz x My x Mx), inverted as (Sz x Sy x Sx) diag(1 / (h1 (lx_i + ly_j + lz_k)
 * + h2)) (Sz x Sy x Sx)^T (a zero denominator, the constant mode of an element
 * without neighbours under h2 = 0, contributes zero).  S[a] and lam[a] are the
 * 1-D factors of direction a; r, z are n^3 with i fastest. */
int orc_fdm_apply(int N, const double *Sx, const double *lx, const double *Sy, const double *ly,
                  const double *Sz, const double *lz, double h1, double h2, const double *r, double *z)
{
    int n = N + 1, n3 = n * n * n;
    double *t = malloc(sizeof(double) * 2 * n3), *u = t + n3;
    const double *S[3] = {Sx, Sy, Sz};
    /* t = (S^T x S^T x S^T) r, one direction at a time */
    memcpy(t, r, sizeof(double) * n3);
    for (int a = 0; a < 3; ++a) {
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    int idx[3] = {i, j, k};
                    double s = 0;
                    for (int l = 0; l < n; ++l) {
                        int m[3] = {i, j, k};
                        m[a] = l;
                        s += S[a][l * n + idx[a]] * t[(m[2] * n + m[1]) * n + m[0]];
                    }
                    u[(k * n + j) * n + i] = s;
                }
        memcpy(t, u, sizeof(double) * n3);
    }
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double d = h1 * (lx[i] + ly[j] + lz[k]) + h2;
                t[(k * n + j) * n + i] = d != 0.0 ? t[(k * n + j) * n + i] / d : 0.0;
            }
    /* z = (S x S x S) t */
    for (int a = 0; a < 3; ++a) {
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    int idx[3] = {i, j, k};
                    double s = 0;
                    for (int l = 0; l < n; ++l) {
                        int m[3] = {i, j, k};
                        m[a] = l;
                        s += S[a][idx[a] * n + l] * t[(m[2] * n + m[1]) * n + m[0]];
                    }
                    u[(k * n + j) * n + i] = s;
                }
        memcpy(t, u, sizeof(double) * n3);
    }
    memcpy(z, t, sizeof(double) * n3);
    free(t);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The multigrid hierarchy                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, n, n3;
    size_t nL;
    double D[(ORC_NMAX + 1) * (ORC_NMAX + 1)];
    double *G, *B, *mult, *imult;
    double *S, *lam;  /* per element and direction: S[(e*3 + a)*n*n], lam[(e*3 + a)*n] */
} orc_level;

typedef struct {
    int nlev, nelx, nely, nelz, periodic[3];
    long E;
    double h1, h2, ctol;
    int cmaxit;
    orc_level L[3];
    double *J[2];     /* J[l]: (n_l x n_{l+1}) interpolation from level l+1 to level l */
    double cstat[2];  /* coarse solves made, coarse iterations summed */
} orc_hsmg;

/* Element lengths along each direction (mean of the four edges). */
static void elem_lengths(int nelx, int nely, const double *vert, long e, double h[3])
{
    int ex = (int)(e % nelx), ey = (int)((e / nelx) % nely), ez = (int)(e / ((long)nelx * nely));
    for (int a = 0; a < 3; ++a) {
        double s = 0;
        for (int c0 = 0; c0 < 2; ++c0)
            for (int c1 = 0; c1 < 2; ++c1) {
                int lo[3], hi[3];
                /* the two corners of the edge along a with the other two offsets (c0, c1) */
                int o[3];
                int b0 = (a + 1) % 3, b1 = (a + 2) % 3;
                o[a] = 0; o[b0] = c0; o[b1] = c1;
                lo[0] = ex + o[0]; lo[1] = ey + o[1]; lo[2] = ez + o[2];
                o[a] = 1;
                hi[0] = ex + o[0]; hi[1] = ey + o[1]; hi[2] = ez + o[2];
                size_t vl = ((size_t)lo[2] * (nely + 1) + lo[1]) * (nelx + 1) + lo[0];
                size_t vh = ((size_t)hi[2] * (nely + 1) + hi[1]) * (nelx + 1) + hi[0];
                double d2 = 0;
                for (int c = 0; c < 3; ++c) {
                    double d = vert[vh * 3 + c] - vert[vl * 3 + c];
                    d2 += d * d;
                }
                s += sqrt(d2);
            }
        h[a] = 0.25 * s;
    }
}

void orc_hsmg_destroy(void *hnd)
{
    orc_hsmg *H = hnd;
    if (!H) return;
    for (int l = 0; l < 3; ++l) {
        free(H->L[l].G);
        free(H->L[l].S);
    }
    free(H->J[0]);
    free(H->J[1]);
    free(H);
}

/* Hierarchy of nlev (1..3) levels of orders orders[0] > orders[1] > ... on the
 * mesh (vertices as for orc_geom), for the operator h1 A + h2 B; the coarsest
 * level is solved by Jacobi-PCG to relative tolerance ctol within cmaxit
 * iterations. */
void *orc_hsmg_create(int nlev, const int *orders, int nelx, int nely, int nelz, const int *periodic,
                      const double *vert, double h1, double h2, double ctol, int cmaxit)
{
    if (nlev < 1 || nlev > 3) return NULL;
    for (int l = 0; l < nlev; ++l)
        if (orders[l] < 1 || orders[l] > ORC_NMAX || (l > 0 && orders[l] >= orders[l - 1])) return NULL;
    orc_hsmg *H = calloc(1, sizeof(orc_hsmg));
    H->nlev = nlev;
    H->nelx = nelx; H->nely = nely; H->nelz = nelz;
    for (int a = 0; a < 3; ++a) H->periodic[a] = periodic[a];
    H->E = (long)nelx * nely * nelz;
    H->h1 = h1; H->h2 = h2; H->ctol = ctol; H->cmaxit = cmaxit;
    int nel[3] = {nelx, nely, nelz};
    for (int l = 0; l < nlev; ++l) {
        orc_level *L = &H->L[l];
        L->N = orders[l];
        L->n = L->N + 1;
        L->n3 = L->n * L->n * L->n;
        L->nL = (size_t)H->E * L->n3;
        double xi[ORC_NMAX + 1], w[ORC_NMAX + 1];
        orc_gll(L->N, xi, w);
        orc_deriv(L->N, xi, L->D);
        L->G = malloc(sizeof(double) * 9 * L->nL);
        L->B = L->G + 6 * L->nL;
        L->mult = L->B + L->nL;
        L->imult = L->mult + L->nL;
        orc_geom(L->N, nelx, nely, nelz, vert, NULL, NULL, L->G, L->B);
        orc_mult(L->N, nelx, nely, nelz, periodic, L->mult);
        for (size_t q = 0; q < L->nL; ++q) L->imult[q] = 1.0 / L->mult[q];
        if (l == nlev - 1) continue;  /* the coarsest level is solved, not smoothed */
        int n = L->n;
        L->S = malloc(sizeof(double) * H->E * 3 * (n * n + n));
        L->lam = L->S + H->E * 3 * n * n;
        for (long e = 0; e < H->E; ++e) {
            long ec[3] = {e % nelx, (e / nelx) % nely, e / ((long)nelx * nely)};
            double h[3];
            elem_lengths(nelx, nely, vert, e, h);
            for (int a = 0; a < 3; ++a) {
                double hn[2] = {0, 0};
                for (int side = 0; side < 2; ++side) {
                    long c = ec[a] + (side ? 1 : -1);
                    if (c < 0 || c >= nel[a]) {
                        if (!periodic[a]) continue;
                        c = (c + nel[a]) % nel[a];
                    }
                    long en[3] = {ec[0], ec[1], ec[2]};
                    en[a] = c;
                    double hh[3];
                    elem_lengths(nelx, nely, vert, en[0] + nelx * (en[1] + (long)nely * en[2]), hh);
                    hn[side] = hh[a];
                }
                orc_fdm_1d(L->N, h[a], hn[0], hn[1], L->S + (e * 3 + a) * n * n, L->lam + (e * 3 + a) * n,
                           NULL, NULL);
            }
        }
    }
    for (int l = 0; l + 1 < nlev; ++l) {
        double xf[ORC_NMAX + 1], xc[ORC_NMAX + 1], w[ORC_NMAX + 1];
        orc_gll(H->L[l].N, xf, w);
        orc_gll(H->L[l + 1].N, xc, w);
        H->J[l] = malloc(sizeof(double) * H->L[l].n * H->L[l + 1].n);
        orc_interp(H->L[l + 1].N, xc, H->L[l].n, xf, H->J[l]);
    }
    return H;
}

/* A_l x (assembled) */
static void level_A(const orc_hsmg *H, int l, const double *x, double *y)
{
    const orc_level *L = &H->L[l];
    orc_ax(L->N, H->E, L->D, L->G, L->B, H->h1, H->h2, x, y);
    orc_dssum(L->N, H->nelx, H->nely, H->nelz, H->periodic, y);
}

/* Schwarz smoother of level l: z = dssum(W sum_e A~_e^{-1} r_e). */
static void smooth(const orc_hsmg *H, int l, const double *r, double *z)
{
    const orc_level *L = &H->L[l];
    int n = L->n, n3 = L->n3;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < H->E; ++e) {
        const double *S = L->S + e * 3 * n * n, *lam = L->lam + e * 3 * n;
        orc_fdm_apply(L->N, S, lam, S + n * n, lam + n, S + 2 * n * n, lam + 2 * n, H->h1, H->h2,
                      r + (size_t)e * n3, z + (size_t)e * n3);
        for (int p = 0; p < n3; ++p) z[(size_t)e * n3 + p] *= L->imult[(size_t)e * n3 + p];
    }
    orc_dssum(L->N, H->nelx, H->nely, H->nelz, H->periodic, z);
}

/* Tensor interpolation on every element: out (level l, n_l^3) = (J x J x J) in
 * (level l+1), or its transpose (trans != 0: in level l, out level l+1). */
static void transfer(const orc_hsmg *H, int l, int trans, const double *in, double *out)
{
    int nf = H->L[l].n, nc = H->L[l + 1].n;
    int ni = trans ? nf : nc, no = trans ? nc : nf;
    const double *J = H->J[l];
#pragma omp parallel for schedule(static)
    for (long e = 0; e < H->E; ++e) {
        const double *u = in + (size_t)e * ni * ni * ni;
        double *v = out + (size_t)e * no * no * no;
        for (int k = 0; k < no; ++k)
            for (int j = 0; j < no; ++j)
                for (int i = 0; i < no; ++i) {
                    double s = 0;
                    for (int c = 0; c < ni; ++c)
                        for (int b = 0; b < ni; ++b)
                            for (int a = 0; a < ni; ++a) {
                                double wgt = trans ? J[a * nc + i] * J[b * nc + j] * J[c * nc + k]
                                                   : J[i * nc + a] * J[j * nc + b] * J[k * nc + c];
                                s += wgt * u[(c * ni + b) * ni + a];
                            }
                    v[(k * no + j) * no + i] = s;
                }
    }
}

/* Prolongation (level l+1 -> l, continuous fields). */
int orc_hsmg_prolong(void *hnd, int l, const double *in, double *out)
{
    orc_hsmg *H = hnd;
    if (l < 0 || l + 1 >= H->nlev) return ORC_ERR_ARG;
    transfer(H, l, 0, in, out);
    return ORC_OK;
}

/* Restriction of a residual (level l -> l+1): dssum(J^T (r / mult_l)). */
int orc_hsmg_restrict(void *hnd, int l, const double *in, double *out)
{
    orc_hsmg *H = hnd;
    if (l < 0 || l + 1 >= H->nlev) return ORC_ERR_ARG;
    size_t nL = H->L[l].nL;
    double *t = malloc(sizeof(double) * nL);
    for (size_t q = 0; q < nL; ++q) t[q] = in[q] * H->L[l].imult[q];
    transfer(H, l, 1, t, out);
    orc_dssum(H->L[l + 1].N, H->nelx, H->nely, H->nelz, H->periodic, out);
    free(t);
    return ORC_OK;
}

/* One V-cycle from level l: z = M_l^{-1} r. */
static void vcycle(orc_hsmg *H, int l, const double *r, double *z)
{
    const orc_level *L = &H->L[l];
    if (l == H->nlev - 1) {
        double out[3];
        memset(z, 0, sizeof(double) * L->nL);
        orc_pcg(L->N, H->nelx, H->nely, H->nelz, H->periodic, L->D, L->G, L->B, H->h1, H->h2, r, z,
                H->ctol, 0, H->cmaxit, out);
        H->cstat[0] += 1;
        H->cstat[1] += out[0];
        return;
    }
    const orc_level *C = &H->L[l + 1];
    double *w = malloc(sizeof(double) * (L->nL + 2 * C->nL)), *rc = w + L->nL, *zc = rc + C->nL;
    smooth(H, l, r, z);
    level_A(H, l, z, w);
    for (size_t q = 0; q < L->nL; ++q) w[q] = r[q] - w[q];
    orc_hsmg_restrict(H, l, w, rc);
    vcycle(H, l + 1, rc, zc);
    transfer(H, l, 0, zc, w);
    for (size_t q = 0; q < L->nL; ++q) z[q] += w[q];
    free(w);
}

/* z = M^{-1} r (one V-cycle from the finest level). */
int orc_hsmg_apply(void *hnd, const double *r, double *z)
{
    vcycle((orc_hsmg *)hnd, 0, r, z);
    return ORC_OK;
}

/* Smoother of level l alone (for tests). */
int orc_hsmg_smooth(void *hnd, int l, const double *r, double *z)
{
    orc_hsmg *H = hnd;
    if (l < 0 || l >= H->nlev - 1) return ORC_ERR_ARG;
    smooth(H, l, r, z);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Flexible GMRES (Saad 1993), right preconditioned, restarted               */
/* ------------------------------------------------------------------------ */

/* Solve dssum(h1 A + h2 B) x = b on the finest level of H (or, with hnd ==
 * NULL, on the order-N mesh given by N, D, G, B with no preconditioner).
 * Stopping test ||b - A x|| <= tol (abs_tol) or tol ||b||, met by the true
 * assembled residual at a restart or by the Arnoldi estimate inside a cycle
 * (the usual GMRES test; out[1] reports the true residual).  With h2 == 0 b loses its mean first and x its
 * B-weighted mean at the end, as in orc_pcg.  out[0] = iterations, out[1] =
 * final true ||r||, out[2] = ||b||, out[3] = restarts; hist (may be NULL,
 * maxit + 1 entries) receives the Arnoldi residual estimate after each
 * iteration (hist[0] = initial residual). */
int orc_fgmres(void *hnd, int N, int nelx, int nely, int nelz, const int *periodic, const double *Dm,
               const double *Gm, const double *Bm, double h1, double h2, const double *b_in, double *x,
               double tol, int abs_tol, int m, int maxit, double *out, double *hist)
{
    orc_hsmg *H = hnd;
    if (H) {
        N = H->L[0].N; nelx = H->nelx; nely = H->nely; nelz = H->nelz; periodic = H->periodic;
        Dm = H->L[0].D; Gm = H->L[0].G; Bm = H->L[0].B; h1 = H->h1; h2 = H->h2;
    }
    if (m < 1 || maxit < 0) return ORC_ERR_ARG;
    int n3 = (N + 1) * (N + 1) * (N + 1);
    long E = (long)nelx * nely * nelz;
    size_t nL = (size_t)E * n3;
    double *mult = malloc(sizeof(double) * nL * 4), *imult = mult + nL, *b = imult + nL, *r = b + nL;
    orc_mult(N, nelx, nely, nelz, periodic, mult);
    for (size_t q = 0; q < nL; ++q) imult[q] = 1.0 / mult[q];
    memcpy(b, b_in, sizeof(double) * nL);
    int singular = (h2 == 0.0);
    if (singular) {
        double sb = 0, s1 = 0;
        for (size_t q = 0; q < nL; ++q) { sb += b[q] * imult[q]; s1 += imult[q]; }
        double mb = sb / s1;
        for (size_t q = 0; q < nL; ++q) b[q] -= mb;
    }
    double *V = malloc(sizeof(double) * nL * (2 * m + 2)), *Z = V + nL * (m + 1), *w = Z + nL * m;
    double *Hs = calloc((size_t)(m + 1) * m, sizeof(double)), *cs = malloc(sizeof(double) * 3 * (m + 1));
    double *sn = cs + (m + 1), *g = sn + (m + 1);
#define AOP(xx, yy)                                                   \
    do {                                                              \
        orc_ax(N, E, Dm, Gm, Bm, h1, h2, (xx), (yy));                 \
        orc_dssum(N, nelx, nely, nelz, periodic, (yy));               \
    } while (0)
    double bnorm = sqrt(orc_glsc3(E, n3, b, b, imult));
    double target = abs_tol ? tol : tol * bnorm;
    AOP(x, w);
    for (size_t q = 0; q < nL; ++q) r[q] = b[q] - w[q];
    double beta = sqrt(orc_glsc3(E, n3, r, r, imult));
    if (hist) hist[0] = beta;
    int it = 0, restarts = 0, status = ORC_ERR_NOT_CONVERGED, met = 0;
    if (!isfinite(beta)) status = ORC_ERR_BREAKDOWN;
    else if (beta <= target) status = ORC_OK;
    while (status == ORC_ERR_NOT_CONVERGED && it < maxit) {
        for (size_t q = 0; q < nL; ++q) V[q] = r[q] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m && it < maxit; ++j) {
            double *vj = V + nL * j, *zj = Z + nL * j;
            if (H) orc_hsmg_apply(H, vj, zj);
            else memcpy(zj, vj, sizeof(double) * nL);
            AOP(zj, w);
            for (int i = 0; i <= j; ++i) {  /* modified Gram-Schmidt */
                double hij = orc_glsc3(E, n3, w, V + nL * i, imult);
                Hs[i * m + j] = hij;
                for (size_t q = 0; q < nL; ++q) w[q] -= hij * V[nL * i + q];
            }
            double hn = sqrt(orc_glsc3(E, n3, w, w, imult));
            for (int i = 0; i < j; ++i) {  /* previous rotations on column j */
                double a = Hs[i * m + j], c = Hs[(i + 1) * m + j];
                Hs[i * m + j] = cs[i] * a + sn[i] * c;
                Hs[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = Hs[j * m + j], rho = sqrt(a * a + hn * hn);
            if (!(rho > 0) || !isfinite(rho)) { status = ORC_ERR_BREAKDOWN; k = j; break; }
            cs[j] = a / rho;
            sn[j] = hn / rho;
            Hs[j * m + j] = rho;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            k = j + 1;
            if (hist) hist[it] = fabs(g[j + 1]);
            if (fabs(g[j + 1]) <= target || hn == 0.0) { met = 1; break; }
            for (size_t q = 0; q < nL; ++q) V[nL * (j + 1) + q] = w[q] / hn;
        }
        /* y = R^{-1} g, x += Z y */
        double y[k > 0 ? k : 1];
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int c = i + 1; c < k; ++c) s -= Hs[i * m + c] * y[c];
            y[i] = s / Hs[i * m + i];
        }
        for (int i = 0; i < k; ++i)
            for (size_t q = 0; q < nL; ++q) x[q] += y[i] * Z[nL * i + q];
        AOP(x, w);
        for (size_t q = 0; q < nL; ++q) r[q] = b[q] - w[q];
        beta = sqrt(orc_glsc3(E, n3, r, r, imult));
        if (status == ORC_ERR_BREAKDOWN) break;
        if (!isfinite(beta)) { status = ORC_ERR_BREAKDOWN; break; }
        if (beta <= target || met) { status = ORC_OK; break; }
        ++restarts;
    }
#undef AOP
    if (singular) {
        double sbx = 0, sb = 0;
        for (size_t q = 0; q < nL; ++q) { sbx += Bm[q] * x[q]; sb += Bm[q]; }
        for (size_t q = 0; q < nL; ++q) x[q] -= sbx / sb;
    }
    out[0] = it; out[1] = beta; out[2] = bnorm; out[3] = restarts;
    free(mult); free(V); free(Hs); free(cs);
    return status;
}

/* Coarse solves made and coarse iterations summed since the last call. */
void orc_hsmg_coarse_stats(void *hnd, double *solves, double *iters)
{
    orc_hsmg *H = hnd;
    *solves = H->cstat[0];
    *iters = H->cstat[1];
    H->cstat[0] = H->cstat[1] = 0;
}
