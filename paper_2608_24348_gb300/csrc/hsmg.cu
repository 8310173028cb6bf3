// hsmg.cu -- the pressure solver of the paper: flexible GMRES preconditioned
// by a hybrid Schwarz multigrid (HSMG) whose coarsest problem is solved by CG
// with the Jacobi preconditioner (Sec. 1; Sec. 3 solver settings).
//
// Levels are polynomial orders on one mesh (e.g. N, 3, 1), each with its own
// context (geometry, operator, gather-scatter).  One preconditioner
// application is a V-cycle:
//     z_l = S_l r_l,  w = r_l - A_l z_l,  r_{l+1} = dssum(J^T (w / mult_l)),
//     z_{l+1} = cycle(r_{l+1}),  z_l += J z_{l+1};
// on the coarsest level z = A^{-1} r by the persistent Jacobi-PCG to a relative
// tolerance.  S_l is the overlapping Schwarz smoother
//     S r = dssum( (1/mult) * sum_e A~_e^{-1} r_e ),
// A~_e the separable (box) form of the element operator, extended at each face
// by the linear segment to the neighbour's first interior GLL node with a zero
// value there, inverted by fast diagonalisation:
//     A~^{-1} = (Sz x Sy x Sx) diag(1 / (h1 (lx_i + ly_j + lz_k) + h2)) (Sz x Sy x Sx)^T,
// where K S = M S diag(lam), S^T M S = I for the extended 1-D stiffness K and
// (diagonal) mass M of each direction.  The V-cycle runs in FP32 or FP64; the
// GMRES vectors, its operator (the FP64-accurate one of sem_ax) and its inner
// products (sum_local a b / mult) are FP64.  GMRES is right preconditioned and
// flexible (x = x0 + Z y), restarted after m steps, with classical
// Gram-Schmidt (a second pass where the first cancelled) and Givens
// rotations; the small Hessenberg
// problem is solved on the host, which reads the inner products back each
// iteration.
#include <math.h>
#include <string.h>

#include <array>
#include <map>
#include <vector>

#include "common.cuh"

int sem_dssum_dev(sem_ctx *c, void *u, sem_dtype dt, cudaStream_t s);
int sem_ax_dev(sem_ctx *c, const void *u, void *w, double h1, double h2, sem_dtype dt, cudaStream_t s);
int sem_pcg_solve_dev(sem_ctx *c, int slot, const double *b, double *x, double h1, double h2,
                      const sem_solve_opts &o, cudaStream_t s);

#define HS_MAXLEV 3
#define HS_DOT_BLOCKS 1216  // 8 x 152 SMs; fixed so that the sums are deterministic
#define HS_DOT_K 8          // inner products per pass over the data

// ---------------------------------------------------------------------------
// Host: 1-D factors of the local solves
// ---------------------------------------------------------------------------

// Symmetric eigenproblem A = V diag(d) V^T by Jacobi rotations, each pivot the
// largest remaining off-diagonal entry (classical Jacobi).  A (n x n, row
// major) is overwritten; V[i*n + k] is entry i of eigenvector k.
static void hs_sym_eig(int n, std::vector<double> &A, std::vector<double> &d, std::vector<double> &V)
{
    V.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    double fro = 0.0;
    for (double a : A) fro += a * a;
    for (int iter = 0; iter < 50 * n * n; ++iter) {
        int p = 0, q = 1;
        double big = -1.0;
        for (int i = 0; i < n; ++i)
            for (int k = i + 1; k < n; ++k)
                if (fabs(A[i * n + k]) > big) { big = fabs(A[i * n + k]); p = i; q = k; }
        if (n < 2 || big * big <= 1e-32 * fro) break;
        // rotation angle that zeroes A[p][q]: tan(2 phi) = 2 A_pq / (A_qq - A_pp)
        const double phi = 0.5 * atan2(2.0 * A[p * n + q], A[q * n + q] - A[p * n + p]);
        const double c = cos(phi), s = sin(phi);
        for (int k = 0; k < n; ++k) {
            const double akp = A[k * n + p], akq = A[k * n + q];
            A[k * n + p] = c * akp - s * akq;
            A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
            const double apk = A[p * n + k], aqk = A[q * n + k];
            A[p * n + k] = c * apk - s * aqk;
            A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
            const double vkp = V[k * n + p], vkq = V[k * n + q];
            V[k * n + p] = c * vkp - s * vkq;
            V[k * n + q] = s * vkp + c * vkq;
        }
    }
    d.resize(n);
    for (int i = 0; i < n; ++i) d[i] = A[i * n + i];
}

// Generalised eigenpairs of the extended 1-D operators of an element of length
// h with neighbour lengths hl, hr (0: none):
//   K = (2/h) Kref + diag(1/dl, 0.., 1/dr),  M = (h/2) diag(w) + diag(dl/2, 0.., dr/2),
//   Kref_ij = sum_q w_q D_qi D_qj,  dl = (xi_1 - xi_0) hl / 2  (likewise dr).
static void hs_fdm_1d(const sem_ctx *c, double h, double hl, double hr, double *S, double *lam)
{
    const int n = c->n;
    std::vector<double> K(n * n), M(n), C(n * n), d, V;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += c->hw[q] * c->hD[q * n + i] * c->hD[q * n + j];
            K[i * n + j] = s * (2.0 / h);
        }
    for (int i = 0; i < n; ++i) M[i] = c->hw[i] * (0.5 * h);
    const double gap = c->hxi[1] - c->hxi[0];
    if (hl > 0) {
        K[0] += 2.0 / (gap * hl);
        M[0] += 0.25 * gap * hl;
    }
    if (hr > 0) {
        K[n * n - 1] += 2.0 / (gap * hr);
        M[n - 1] += 0.25 * gap * hr;
    }
    // C = M^{-1/2} K M^{-1/2} = V diag(d) V^T  ->  S = M^{-1/2} V
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) C[i * n + j] = K[i * n + j] / (sqrt(M[i]) * sqrt(M[j]));
    hs_sym_eig(n, C, d, V);
    for (int i = 0; i < n; ++i) {
        lam[i] = d[i];
        for (int k = 0; k < n; ++k) S[i * n + k] = V[i * n + k] / sqrt(M[i]);
    }
}

// Mean edge length of element (ex, ey, ez) along direction a, from host vertices.
static double hs_edge_len(const sem_ctx *c, const double *vert, int ex, int ey, int ez, int a)
{
    double s = 0.0;
    for (int t = 0; t < 4; ++t) {
        int o[3] = {0, 0, 0};
        o[(a + 1) % 3] = t & 1;
        o[(a + 2) % 3] = t >> 1;
        int p[3] = {ex + o[0], ey + o[1], ez + o[2]};
        const size_t v0 = ((size_t)p[2] * (c->nely + 1) + p[1]) * (c->nelx + 1) + p[0];
        p[a] += 1;
        const size_t v1 = ((size_t)p[2] * (c->nely + 1) + p[1]) * (c->nelx + 1) + p[0];
        double d2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double dd = vert[v1 * 3 + k] - vert[v0 * 3 + k];
            d2 += dd * dd;
        }
        s += sqrt(d2);
    }
    return 0.25 * s;
}

// ---------------------------------------------------------------------------
// Device kernels
// ---------------------------------------------------------------------------

// Fast-diagonalisation local solves of every element, weighted by 1/mult:
// z_e = (1/mult) (S x S x S) diag(1/(h1 sum lam + h2)) (S x S x S)^T r_e.
// fidx[e*3 + a] selects element e's factor set of direction a.
template <int NP, typename T>
__global__ void k_hs_fdm(const T *__restrict__ r, T *__restrict__ z, const T *__restrict__ Sf,
                         const T *__restrict__ lamf, const int *__restrict__ fidx,
                         const T *__restrict__ imult, T h1, T h2, int64_t E)
{
    constexpr int N2 = NP * NP, N3 = N2 * NP;
    __shared__ T sS[3][N2], sl[3][NP], su[N3], st[N3];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * N2; t += blockDim.x) {
            const int a = t / N2, q = t - a * N2;
            sS[a][q] = Sf[(size_t)fidx[e * 3 + a] * N2 + q];
        }
        for (int t = threadIdx.x; t < 3 * NP; t += blockDim.x) {
            const int a = t / NP, q = t - a * NP;
            sl[a][q] = lamf[(size_t)fidx[e * 3 + a] * NP + q];
        }
        const int64_t off = e * N3;
        for (int t = threadIdx.x; t < N3; t += blockDim.x) su[t] = r[off + t];
        __syncthreads();
        // forward: (S^T u)_i = sum_l S[l][i] u_l along x, then y, then z
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % NP, jk = t - i;
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) s = fma(sS[0][l * NP + i], su[jk + l], s);
            st[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % NP, j = (t / NP) % NP, k = t / N2;
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) s = fma(sS[1][l * NP + j], st[(k * NP + l) * NP + i], s);
            su[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % NP, j = (t / NP) % NP, k = t / N2;
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) s = fma(sS[2][l * NP + k], su[(l * NP + j) * NP + i], s);
            const T den = h1 * (sl[0][i] + sl[1][j] + sl[2][k]) + h2;
            st[t] = den != T(0) ? s / den : T(0);
        }
        __syncthreads();
        // backward: (S u)_i = sum_l S[i][l] u_l along z, then y, then x
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % NP, j = (t / NP) % NP, k = t / N2;
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) s = fma(sS[2][k * NP + l], st[(l * NP + j) * NP + i], s);
            su[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % NP, j = (t / NP) % NP, k = t / N2;
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) s = fma(sS[1][j * NP + l], su[(k * NP + l) * NP + i], s);
            st[t] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % NP, jk = t - i;
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) s = fma(sS[0][i * NP + l], st[jk + l], s);
            z[off + t] = s * imult[off + t];
        }
    }
}

// Grid transfer between levels of nf and nc points per direction (nc < nf <= 10).
// prolong (dir 0): out_f = (J x J x J) in_c  (add != 0: out_f += ...);
// restrict (dir 1): out_c = (J^T x J^T x J^T)(in_f / mult_f).
// J[f*nc + c] = l_c(xi_f), the coarse Lagrange basis at the fine GLL points.
#define HS_TMAX 10
template <typename T>
__global__ void k_hs_transfer(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ J,
                              const T *__restrict__ imult_f, int nf, int nc, int dir, int add, int64_t E)
{
    __shared__ T sJ[HS_TMAX * HS_TMAX];
    __shared__ T sa[HS_TMAX * HS_TMAX * HS_TMAX], sb[HS_TMAX * HS_TMAX * HS_TMAX];
    const int ni = dir ? nf : nc, no = dir ? nc : nf;
    const int ni3 = ni * ni * ni, no3 = no * no * no;
    for (int t = threadIdx.x; t < nf * nc; t += blockDim.x) sJ[t] = J[t];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        for (int t = threadIdx.x; t < ni3; t += blockDim.x)
            sa[t] = dir ? in[e * ni3 + t] * imult_f[e * ni3 + t] : in[e * ni3 + t];
        __syncthreads();
        // weight of input point a for output point o along one direction
        auto wgt = [&](int o, int a) -> T { return dir ? sJ[a * nc + o] : sJ[o * nc + a]; };
        // x: sb[c][b][i] (ni * ni * no)
        for (int t = threadIdx.x; t < ni * ni * no; t += blockDim.x) {
            const int i = t % no, cb = t / no;
            T s = 0;
            for (int a = 0; a < ni; ++a) s = fma(wgt(i, a), sa[cb * ni + a], s);
            sb[t] = s;
        }
        __syncthreads();
        // y: sa[c][j][i] (ni * no * no)
        for (int t = threadIdx.x; t < ni * no * no; t += blockDim.x) {
            const int i = t % no, j = (t / no) % no, c = t / (no * no);
            T s = 0;
            for (int b = 0; b < ni; ++b) s = fma(wgt(j, b), sb[(c * ni + b) * no + i], s);
            sa[t] = s;
        }
        __syncthreads();
        // z: out[k][j][i]
        for (int t = threadIdx.x; t < no3; t += blockDim.x) {
            const int ji = t % (no * no), k = t / (no * no);
            T s = 0;
            for (int c = 0; c < ni; ++c) s = fma(wgt(k, c), sa[c * no * no + ji], s);
            out[e * no3 + t] = add ? out[e * no3 + t] + s : s;
        }
    }
}

template <typename T>
__global__ void k_hs_sub(T *__restrict__ w, const T *__restrict__ r, int64_t n)  // w = r - w
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        w[t] = r[t] - w[t];
}

template <typename A, typename B>
__global__ void k_hs_conv(const A *__restrict__ a, B *__restrict__ b, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (B)a[t];
}

__global__ void k_hs_fill(double *a, double v, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        a[t] = v;
}

// Partial inner products <w, v_i> = sum_local w v_i / mult for up to
// HS_DOT_K vectors v_i = V + i*ld (V == nullptr: the constant 1), one row of
// HS_DOT_BLOCKS partials per vector, summed by k_hs_dot_final in a fixed order.
__global__ void k_hs_dots(const double *__restrict__ w, const double *__restrict__ V, int64_t ld, int k,
                          const double *__restrict__ imult, double *__restrict__ part, int64_t n)
{
    double acc[HS_DOT_K];
#pragma unroll
    for (int i = 0; i < HS_DOT_K; ++i) acc[i] = 0.0;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // four grid strides per pass, every load of a pass issued before its use
    for (; t + 3 * G < n; t += 4 * G) {
        double a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = w[t + q * G] * imult[t + q * G];
#pragma unroll
        for (int i = 0; i < HS_DOT_K; ++i)
            if (i < k) {
                double v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = V ? V[i * ld + t + q * G] : 1.0;
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i] = fma(a[q], v[q], acc[i]);
            }
    }
    for (; t < n; t += G) {
        const double a = w[t] * imult[t];
#pragma unroll
        for (int i = 0; i < HS_DOT_K; ++i)
            if (i < k) acc[i] = fma(a, V ? V[i * ld + t] : 1.0, acc[i]);
    }
    __shared__ double red[HS_DOT_K][32];
#pragma unroll
    for (int i = 0; i < HS_DOT_K; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double s = 0.0;
        for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp) s += red[threadIdx.x][wp];
        part[threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

// One block per value: a fixed strided split of the nb partials over the
// threads, then a fixed tree (blockDim.x a power of two).
__global__ void k_hs_dot_final(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    __shared__ double red[256];
    const double *p = part + (size_t)blockIdx.x * nb;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += p[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// y += sum_i c_i v_i for up to 16 vectors v_i = V + i*ld
struct HsCoef {
    double c[16];
};

__global__ void k_hs_maxpy(double *__restrict__ y, const double *__restrict__ V, int64_t ld, int k, HsCoef cf,
                           int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double s = y[t];
        for (int i = 0; i < k; ++i) s = fma(cf.c[i], V[i * ld + t], s);
        y[t] = s;
    }
}

__global__ void k_hs_scale(double *__restrict__ y, const double *__restrict__ x, double a, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] = a * x[t];
}

// sum_local B x and sum_local B (B from the element-blocked geometry).
__global__ void k_hs_bsum(const double *__restrict__ x, const double *__restrict__ geo64, int n3, int64_t E,
                          double *__restrict__ part)
{
    double a = 0.0, b = 0.0;
    const int64_t n = E * n3;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / n3;
        const double bm = geo64[(e * 7 + 6) * n3 + (t - e * n3)];
        a = fma(bm, x[t], a);
        b += bm;
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp) s += red[threadIdx.x][wp];
        part[threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_hs_add_scalar(double *__restrict__ x, double v, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        x[t] += v;
}

// ---------------------------------------------------------------------------
// Host: hierarchy
// ---------------------------------------------------------------------------

struct HsLevel {
    sem_ctx *c;       // the level's context (the caller's on level 0)
    int own;          // this object created c
    void *r, *z, *w;  // level vectors in the V-cycle precision (r, z unused on level 0 for FP64)
    void *imult;      // 1 / multiplicity, V-cycle precision
    void *S, *lam;    // unique factor sets [nset][n*n], [nset][n]
    int *fidx;        // [E][3]
    void *J;          // interpolation from the next coarser level: [n * n_next]
};

struct sem_hsmg {
    int nlev;
    double h1, h2, ctol;
    int cmaxit;
    sem_dtype dt;     // SEM_F32 or SEM_F64: V-cycle precision
    HsLevel L[HS_MAXLEV];
    double *c64[2];   // coarse right-hand side and solution (FP64)
    // GMRES storage (grown on demand)
    int m_cap;
    double *V, *Z, *r, *w, *imult64, *part, *dots;
    double *hdots;    // pinned host mirror of dots
    sem_solve_info last;
};

static size_t hs_tsize(sem_dtype dt) { return dt == SEM_F32 ? sizeof(float) : sizeof(double); }

static unsigned hs_grid(int64_t n)
{
    const int64_t b = sem_ceil_div(n, 256);
    return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

extern "C" void sem_hsmg_destroy(sem_hsmg *H)
{
    if (!H) return;
    cudaDeviceSynchronize();
    for (int l = 0; l < H->nlev; ++l) {
        HsLevel &L = H->L[l];
        cudaFree(L.r); cudaFree(L.z); cudaFree(L.w); cudaFree(L.imult);
        cudaFree(L.S); cudaFree(L.lam); cudaFree(L.fidx); cudaFree(L.J);
        if (L.own) sem_destroy(L.c);
    }
    cudaFree(H->c64[0]); cudaFree(H->c64[1]);
    cudaFree(H->V); cudaFree(H->Z); cudaFree(H->r); cudaFree(H->w); cudaFree(H->imult64);
    cudaFree(H->part); cudaFree(H->dots);
    if (H->hdots) cudaFreeHost(H->hdots);
    free(H);
}

template <typename T>
__global__ void k_hs_inv(const double *__restrict__ m, T *__restrict__ out, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (T)(1.0 / m[t]);
}

// out = 1/multiplicity of c's local nodes, in precision dt (tmp: nL doubles of scratch).
static int hs_imult(sem_ctx *c, void *out, sem_dtype dt, double *tmp, cudaStream_t s)
{
    const int64_t n = c->nL;
    k_hs_fill<<<hs_grid(n), 256, 0, s>>>(tmp, 1.0, n);
    SEM_CHECK_LAUNCH();
    int rc = sem_dssum_dev(c, tmp, SEM_F64, s);
    if (rc) return rc;
    if (dt == SEM_F32) k_hs_inv<float><<<hs_grid(n), 256, 0, s>>>(tmp, (float *)out, n);
    else k_hs_inv<double><<<hs_grid(n), 256, 0, s>>>(tmp, (double *)out, n);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

template <typename T>
static int hs_upload(void **dst, const std::vector<double> &src)
{
    std::vector<T> h(src.begin(), src.end());
    SEM_CUDA(cudaMalloc(dst, sizeof(T) * (h.size() ? h.size() : 1)));
    SEM_CUDA(cudaMemcpy(*dst, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return SEM_OK;
}

// Fast-diagonalisation factors of every element of level L (unique sets shared).
static int hs_factors(sem_hsmg *H, HsLevel &L, const std::vector<double> &vert)
{
    sem_ctx *c = L.c;
    const int n = c->n;
    std::map<std::array<double, 3>, int> sets;
    std::vector<double> S, lam;
    std::vector<int> fidx(c->E * 3);
    const int nel[3] = {c->nelx, c->nely, c->nelz};
    for (int64_t e = 0; e < c->E; ++e) {
        const int ec[3] = {(int)(e % c->nelx), (int)((e / c->nelx) % c->nely), (int)(e / ((int64_t)c->nelx * c->nely))};
        for (int a = 0; a < 3; ++a) {
            std::array<double, 3> key;
            key[0] = hs_edge_len(c, vert.data(), ec[0], ec[1], ec[2], a);
            for (int side = 0; side < 2; ++side) {
                int nb[3] = {ec[0], ec[1], ec[2]};
                nb[a] += side ? 1 : -1;
                double hn = 0.0;
                if (nb[a] < 0 || nb[a] >= nel[a]) {
                    if (c->periodic[a]) {
                        nb[a] = (nb[a] + nel[a]) % nel[a];
                        hn = hs_edge_len(c, vert.data(), nb[0], nb[1], nb[2], a);
                    }
                } else {
                    hn = hs_edge_len(c, vert.data(), nb[0], nb[1], nb[2], a);
                }
                key[1 + side] = hn;
            }
            auto it = sets.find(key);
            int id;
            if (it == sets.end()) {
                id = (int)sets.size();
                sets.emplace(key, id);
                S.resize((size_t)(id + 1) * n * n);
                lam.resize((size_t)(id + 1) * n);
                hs_fdm_1d(c, key[0], key[1], key[2], &S[(size_t)id * n * n], &lam[(size_t)id * n]);
            } else {
                id = it->second;
            }
            fidx[e * 3 + a] = id;
        }
    }
    int rc = H->dt == SEM_F32 ? hs_upload<float>(&L.S, S) : hs_upload<double>(&L.S, S);
    if (!rc) rc = H->dt == SEM_F32 ? hs_upload<float>(&L.lam, lam) : hs_upload<double>(&L.lam, lam);
    if (rc) return rc;
    SEM_CUDA(cudaMalloc(&L.fidx, sizeof(int) * fidx.size()));
    SEM_CUDA(cudaMemcpy(L.fidx, fidx.data(), sizeof(int) * fidx.size(), cudaMemcpyHostToDevice));
    return SEM_OK;
}

extern "C" int sem_hsmg_create(sem_ctx *c, int nlev, const int *orders, double h1, double h2, sem_dtype dt,
                               double coarse_tol, int coarse_maxit, sem_hsmg **out)
{
    if (!out) return SEM_ERR_ARG;
    *out = nullptr;
    if (!c || !orders || nlev < 1 || nlev > HS_MAXLEV || orders[0] != c->N) return SEM_ERR_ARG;
    for (int l = 1; l < nlev; ++l)
        if (orders[l] < 1 || orders[l] >= orders[l - 1]) return SEM_ERR_ARG;
    if (c->n > 10 || (dt != SEM_F32 && dt != SEM_F64) || !(h1 > 0) || !(h2 >= 0) ||
        !(coarse_tol > 0) || coarse_maxit < 1)
        return SEM_ERR_ARG;
    sem_hsmg *H = (sem_hsmg *)calloc(1, sizeof(sem_hsmg));
    if (!H) return SEM_ERR_NOMEM;
    H->nlev = nlev;
    H->h1 = h1; H->h2 = h2; H->ctol = coarse_tol; H->cmaxit = coarse_maxit;
    H->dt = dt;
    int rc = SEM_OK;
#define HS_TRY(x)                          \
    do {                                   \
        rc = (x);                          \
        if (rc) { sem_hsmg_destroy(H); return rc; } \
    } while (0)
#define HS_CU(x)                                                  \
    do {                                                          \
        cudaError_t e_ = (x);                                     \
        if (e_ != cudaSuccess) {                                  \
            sem_note_cuda_error(e_, #x);                          \
            sem_hsmg_destroy(H);                                  \
            return e_ == cudaErrorMemoryAllocation ? SEM_ERR_NOMEM : SEM_ERR_CUDA; \
        }                                                         \
    } while (0)
    // the mesh's vertices on the host, for the coarser contexts and the element lengths
    const size_t nv = (size_t)(c->nelx + 1) * (c->nely + 1) * (c->nelz + 1) * 3;
    std::vector<double> vert(nv);
    HS_CU(cudaMemcpy(vert.data(), c->vert, sizeof(double) * nv, cudaMemcpyDeviceToHost));
    H->L[0].c = c;
    for (int l = 1; l < nlev; ++l) {
        HS_TRY(sem_setup(orders[l], c->nelx, c->nely, c->nelz, c->L, c->periodic, vert.data(), &H->L[l].c));
        H->L[l].own = 1;
    }
    const size_t ts = hs_tsize(dt);
    double *tmp = nullptr;
    HS_CU(cudaMalloc(&tmp, sizeof(double) * c->nL));
    for (int l = 0; l < nlev; ++l) {
        HsLevel &L = H->L[l];
        const int64_t n = L.c->nL;
        HS_CU(cudaMalloc(&L.r, ts * n));
        HS_CU(cudaMalloc(&L.z, ts * n));
        HS_CU(cudaMalloc(&L.w, ts * n));
        HS_CU(cudaMalloc(&L.imult, ts * n));
        rc = hs_imult(L.c, L.imult, dt, tmp, 0);
        if (rc) { cudaFree(tmp); sem_hsmg_destroy(H); return rc; }
        if (l < nlev - 1) {
            rc = hs_factors(H, L, vert);
            if (rc) { cudaFree(tmp); sem_hsmg_destroy(H); return rc; }
            // interpolation from level l+1's GLL points to level l's
            const sem_ctx *cc = H->L[l + 1].c;
            const int nf = L.c->n, nc = cc->n;
            std::vector<double> J((size_t)nf * nc);
            for (int f = 0; f < nf; ++f)
                for (int a = 0; a < nc; ++a) {
                    double v = 1.0;
                    for (int b = 0; b < nc; ++b)
                        if (b != a) v *= (L.c->hxi[f] - cc->hxi[b]) / (cc->hxi[a] - cc->hxi[b]);
                    J[(size_t)f * nc + a] = v;
                }
            rc = dt == SEM_F32 ? hs_upload<float>(&L.J, J) : hs_upload<double>(&L.J, J);
            if (rc) { cudaFree(tmp); sem_hsmg_destroy(H); return rc; }
        }
    }
    // FP64 1/mult of the finest level (GMRES inner products)
    HS_CU(cudaMalloc(&H->imult64, sizeof(double) * c->nL));
    rc = hs_imult(c, H->imult64, SEM_F64, tmp, 0);
    cudaFree(tmp);
    if (rc) { sem_hsmg_destroy(H); return rc; }
    const int64_t ncl = H->L[nlev - 1].c->nL;
    HS_CU(cudaMalloc(&H->c64[0], sizeof(double) * ncl));
    HS_CU(cudaMalloc(&H->c64[1], sizeof(double) * ncl));
    HS_CU(cudaMalloc(&H->part, sizeof(double) * HS_DOT_BLOCKS * HS_DOT_K));
    HS_CU(cudaMalloc(&H->dots, sizeof(double) * 64));
    HS_CU(cudaMallocHost(&H->hdots, sizeof(double) * 64));
    HS_CU(cudaDeviceSynchronize());
#undef HS_TRY
#undef HS_CU
    *out = H;
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// V-cycle
// ---------------------------------------------------------------------------

template <typename T>
static int hs_fdm(sem_hsmg *H, HsLevel &L, const T *r, T *z, cudaStream_t s)
{
    sem_ctx *c = L.c;
    const int n3 = c->n * c->n * c->n;
    const int threads = n3 >= 256 ? 256 : ((n3 + 31) / 32) * 32;
    const int64_t grid64 = c->E < (int64_t)c->num_sms * 16 ? c->E : (int64_t)c->num_sms * 16;
    const unsigned grid = (unsigned)(grid64 > 0 ? grid64 : 1);
#define HS_FDM_CASE(NPV)                                                                          \
    case NPV:                                                                                     \
        k_hs_fdm<NPV, T><<<grid, threads, 0, s>>>(r, z, (const T *)L.S, (const T *)L.lam, L.fidx, \
                                                   (const T *)L.imult, (T)H->h1, (T)H->h2, c->E); \
        break;
    switch (c->n) {
        HS_FDM_CASE(2) HS_FDM_CASE(3) HS_FDM_CASE(4) HS_FDM_CASE(5) HS_FDM_CASE(6)
        HS_FDM_CASE(7) HS_FDM_CASE(8) HS_FDM_CASE(9) HS_FDM_CASE(10)
        default: return SEM_ERR_ARG;
    }
#undef HS_FDM_CASE
    SEM_CHECK_LAUNCH();
    return sem_dssum_dev(c, z, H->dt, s);
}

template <typename T>
static int hs_transfer(sem_hsmg *H, int l, const T *in, T *out, int dir, int add, cudaStream_t s)
{
    HsLevel &L = H->L[l];
    const sem_ctx *cf = L.c, *cc = H->L[l + 1].c;
    const unsigned grid = (unsigned)(cf->E < (int64_t)cf->num_sms * 16 ? cf->E : (int64_t)cf->num_sms * 16);
    k_hs_transfer<T><<<grid > 0 ? grid : 1, 128, 0, s>>>(in, out, (const T *)L.J, (const T *)L.imult, cf->n,
                                                         cc->n, dir, add, cf->E);
    SEM_CHECK_LAUNCH();
    if (dir) return sem_dssum_dev(H->L[l + 1].c, out, H->dt, s);
    return SEM_OK;
}

// z = M_l^{-1} r on level l (r, z: level vectors in the V-cycle precision).
template <typename T>
static int hs_cycle(sem_hsmg *H, int l, T *r, T *z, cudaStream_t s)
{
    HsLevel &L = H->L[l];
    sem_ctx *c = L.c;
    const int64_t n = c->nL;
    int rc;
    if (l == H->nlev - 1) {  // coarsest: Jacobi-PCG in FP64 from a zero guess
        k_hs_conv<T, double><<<hs_grid(n), 256, 0, s>>>(r, H->c64[0], n);
        SEM_CHECK_LAUNCH();
        SEM_CUDA(cudaMemsetAsync(H->c64[1], 0, sizeof(double) * n, s));
        sem_solve_opts o;
        sem_solve_opts_default(&o);
        o.tol = H->ctol;
        o.abs_tol = 0;
        o.maxit = H->cmaxit;
        if ((rc = sem_pcg_solve_dev(c, 0, H->c64[0], H->c64[1], H->h1, H->h2, o, s))) return rc;
        k_hs_conv<double, T><<<hs_grid(n), 256, 0, s>>>(H->c64[1], z, n);
        SEM_CHECK_LAUNCH();
        return SEM_OK;
    }
    HsLevel &C = H->L[l + 1];
    T *w = (T *)L.w;
    if ((rc = hs_fdm<T>(H, L, r, z, s))) return rc;
    if ((rc = sem_ax_dev(c, z, w, H->h1, H->h2, H->dt, s))) return rc;
    if ((rc = sem_dssum_dev(c, w, H->dt, s))) return rc;
    k_hs_sub<T><<<hs_grid(n), 256, 0, s>>>(w, r, n);
    SEM_CHECK_LAUNCH();
    if ((rc = hs_transfer<T>(H, l, w, (T *)C.r, 1, 0, s))) return rc;
    if ((rc = hs_cycle<T>(H, l + 1, (T *)C.r, (T *)C.z, s))) return rc;
    return hs_transfer<T>(H, l, (const T *)C.z, z, 0, 1, s);
}

// z = M^{-1} r for FP64 E-vectors of the finest level.
static int hs_apply_dev(sem_hsmg *H, const double *r, double *z, cudaStream_t s)
{
    const int64_t n = H->L[0].c->nL;
    if (H->dt == SEM_F32) {
        k_hs_conv<double, float><<<hs_grid(n), 256, 0, s>>>(r, (float *)H->L[0].r, n);
        SEM_CHECK_LAUNCH();
        int rc = hs_cycle<float>(H, 0, (float *)H->L[0].r, (float *)H->L[0].z, s);
        if (rc) return rc;
        k_hs_conv<float, double><<<hs_grid(n), 256, 0, s>>>((const float *)H->L[0].z, z, n);
        SEM_CHECK_LAUNCH();
        return SEM_OK;
    }
    return hs_cycle<double>(H, 0, (double *)r, z, s);
}

extern "C" int sem_hsmg_apply(sem_hsmg *H, const double *r, double *z, void *stream)
{
    if (!H || !r || !z || !sem_is_device_ptr(r) || !sem_is_device_ptr(z)) return SEM_ERR_ARG;
    return hs_apply_dev(H, r, z, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Flexible GMRES
// ---------------------------------------------------------------------------

// dots[i] = <w, v_i>, i < k (V == nullptr: <w, 1>), into H->hdots (synchronises s).
// (enqueue only: the values land in H->dots + at)
static int hs_dots_enq(sem_hsmg *H, const double *w, const double *V, int64_t ld, int k, int at, cudaStream_t s)
{
    const int64_t n = H->L[0].c->nL;
    for (int i0 = 0; i0 < k; i0 += HS_DOT_K) {
        const int kk = k - i0 < HS_DOT_K ? k - i0 : HS_DOT_K;
        k_hs_dots<<<HS_DOT_BLOCKS, 256, 0, s>>>(w, V ? V + i0 * ld : nullptr, ld, kk, H->imult64, H->part, n);
        k_hs_dot_final<<<kk, 256, 0, s>>>(H->part, HS_DOT_BLOCKS, H->dots + at + i0);
        SEM_CHECK_LAUNCH();
    }
    return SEM_OK;
}

static int hs_dots_read(sem_hsmg *H, int k, cudaStream_t s)
{
    SEM_CUDA(cudaMemcpyAsync(H->hdots, H->dots, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
}

static int hs_dots(sem_hsmg *H, const double *w, const double *V, int64_t ld, int k, cudaStream_t s)
{
    int rc = hs_dots_enq(H, w, V, ld, k, 0, s);
    return rc ? rc : hs_dots_read(H, k, s);
}

// y += sum_i c[i] v_i
static int hs_maxpy(sem_hsmg *H, double *y, const double *V, int64_t ld, int k, const double *c, cudaStream_t s)
{
    const int64_t n = H->L[0].c->nL;
    for (int i0 = 0; i0 < k; i0 += 16) {
        const int kk = k - i0 < 16 ? k - i0 : 16;
        HsCoef cf;
        for (int i = 0; i < kk; ++i) cf.c[i] = c[i0 + i];
        k_hs_maxpy<<<hs_grid(n), 256, 0, s>>>(y, V + i0 * ld, ld, kk, cf, n);
        SEM_CHECK_LAUNCH();
    }
    return SEM_OK;
}

static int hs_ensure(sem_hsmg *H, int m)
{
    if (m <= H->m_cap) return SEM_OK;
    const int64_t n = H->L[0].c->nL;
    cudaFree(H->V); cudaFree(H->Z); cudaFree(H->r); cudaFree(H->w);
    H->V = H->Z = H->r = H->w = nullptr;
    H->m_cap = 0;
    cudaError_t e = cudaMalloc(&H->V, sizeof(double) * n * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&H->Z, sizeof(double) * n * m);
    if (e == cudaSuccess) e = cudaMalloc(&H->r, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&H->w, sizeof(double) * n);
    if (e != cudaSuccess) {
        sem_note_cuda_error(e, "cudaMalloc(GMRES basis)");
        return e == cudaErrorMemoryAllocation ? SEM_ERR_NOMEM : SEM_ERR_CUDA;
    }
    H->m_cap = m;
    return SEM_OK;
}

// A x (assembled) with the operator that the tolerance asks for.
static int hs_op(sem_hsmg *H, const double *x, double *y, bool tight, cudaStream_t s)
{
    sem_ctx *c = H->L[0].c;
    int rc = sem_ax_dev(c, x, y, H->h1, H->h2, tight ? SEM_F64_NATIVE : SEM_F64, s);
    if (rc) return rc;
    return sem_dssum_dev(c, y, SEM_F64, s);
}

// x_zero != 0: the caller guarantees x = 0 on entry (the first residual is b').
int sem_gmres_solve_dev(sem_hsmg *H, int precond, const double *b_in, double *x, const sem_solve_opts &o,
                        int m, sem_solve_info *info, cudaStream_t s, int x_zero)
{
    sem_ctx *c = H->L[0].c;
    const int64_t n = c->nL;
    memset(info, 0, sizeof(*info));
    if (m < 1 || m > 64 || !(o.tol >= 0) || o.maxit < 0) return SEM_ERR_ARG;
    int rc = hs_ensure(H, m);
    if (rc) return rc;
    // the plain FP64 operator for tolerances below what the FP32-pipe operators resolve
    const bool tight = !o.abs_tol && o.tol < 1e-11;
    const bool singular = H->h2 == 0.0;
    double *r = H->r, *w = H->w, *V = H->V, *Z = H->Z;
    // b' = b minus its mean over unique nodes when the operator is singular (r holds b')
    SEM_CUDA(cudaMemcpyAsync(r, b_in, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double bmean = 0.0;
    if (singular) {
        if ((rc = hs_dots(H, r, nullptr, 0, 1, s))) return rc;
        bmean = H->hdots[0] / (double)c->nG;
        k_hs_add_scalar<<<hs_grid(n), 256, 0, s>>>(r, -bmean, n);
        SEM_CHECK_LAUNCH();
    }
    if ((rc = hs_dots(H, r, r, n, 1, s))) return rc;
    const double bnorm = sqrt(H->hdots[0]);
    const double target = o.abs_tol ? o.tol : o.tol * bnorm;
    // The true residual decides convergence.  Below 1e-8 ||b|| it is taken
    // with the native FP64 operator: the FP64-accurate operator's rounding
    // floor (a few 1e-13 relative per application, times ||A|| ||x||) can
    // reach that level, and GMRES cycles on the fast operator then act as the
    // inner solves of an FP64 refinement.
    const bool native_res = tight || target < 1e-8 * bnorm;
    auto true_residual = [&](double *beta) -> int {
        // r = b' - A x
        int rc2 = hs_op(H, x, w, native_res, s);
        if (rc2) return rc2;
        SEM_CUDA(cudaMemcpyAsync(r, b_in, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if (singular) {
            k_hs_add_scalar<<<hs_grid(n), 256, 0, s>>>(r, -bmean, n);
            SEM_CHECK_LAUNCH();
        }
        k_hs_sub<double><<<hs_grid(n), 256, 0, s>>>(w, r, n);  // w = r - w
        SEM_CHECK_LAUNCH();
        SEM_CUDA(cudaMemcpyAsync(r, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if ((rc2 = hs_dots(H, r, r, n, 1, s))) return rc2;
        *beta = sqrt(H->hdots[0]);
        return SEM_OK;
    };
    double beta = bnorm;  // x = 0: the first residual is b' (already in r)
    if (!x_zero && (rc = true_residual(&beta))) return rc;
    int it = 0, restarts = 0, status = SEM_ERR_NOT_CONVERGED;
    if (!isfinite(beta) || !isfinite(bnorm)) status = SEM_ERR_BREAKDOWN;
    else if (beta <= target) status = SEM_OK;
    std::vector<double> Hm((size_t)(m + 1) * m), cs(m + 1), sn(m + 1), g(m + 1), y(m), h(m + 1);
    bool estimate_met = false;
    while (status == SEM_ERR_NOT_CONVERGED && it < o.maxit) {
        const double beta0 = beta;
        estimate_met = false;
        k_hs_scale<<<hs_grid(n), 256, 0, s>>>(V, r, 1.0 / beta, n);
        SEM_CHECK_LAUNCH();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        bool broke = false;
        for (int j = 0; j < m && it < o.maxit; ++j) {
            double *vj = V + (int64_t)j * n, *zj = Z + (int64_t)j * n;
            if (precond) {
                if ((rc = hs_apply_dev(H, vj, zj, s))) return rc;
            } else {
                SEM_CUDA(cudaMemcpyAsync(zj, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            }
            if ((rc = hs_op(H, zj, w, tight, s))) return rc;
            // classical Gram-Schmidt; a second pass only when the first removed
            // more than half of |w|^2 ("twice is enough": the first pass's
            // projections lost accuracy to cancellation)
            std::fill(h.begin(), h.end(), 0.0);
            double hn = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                if ((rc = hs_dots_enq(H, w, V, n, j + 1, 0, s))) return rc;
                if ((rc = hs_dots_enq(H, w, w, n, 1, j + 1, s))) return rc;
                if ((rc = hs_dots_read(H, j + 2, s))) return rc;
                const double ww = H->hdots[j + 1];
                std::vector<double> neg(j + 1);
                double proj = 0.0;
                for (int i = 0; i <= j; ++i) {
                    h[i] += H->hdots[i];
                    neg[i] = -H->hdots[i];
                    proj += H->hdots[i] * H->hdots[i];
                }
                if ((rc = hs_maxpy(H, w, V, n, j + 1, neg.data(), s))) return rc;
                if (ww - proj > 0.5 * ww) break;
            }
            if ((rc = hs_dots(H, w, w, n, 1, s))) return rc;
            hn = sqrt(H->hdots[0]);
            for (int i = 0; i <= j; ++i) Hm[(size_t)i * m + j] = h[i];
            for (int i = 0; i < j; ++i) {  // earlier rotations on column j
                const double a = Hm[(size_t)i * m + j], b2 = Hm[(size_t)(i + 1) * m + j];
                Hm[(size_t)i * m + j] = cs[i] * a + sn[i] * b2;
                Hm[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b2;
            }
            const double a = Hm[(size_t)j * m + j], rho = hypot(a, hn);
            if (!(rho > 0) || !isfinite(rho)) { status = SEM_ERR_BREAKDOWN; broke = true; k = j; break; }
            cs[j] = a / rho;
            sn[j] = hn / rho;
            Hm[(size_t)j * m + j] = rho;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            k = j + 1;
            if (fabs(g[j + 1]) <= target || hn == 0.0) {
                estimate_met = true;
                break;
            }
            k_hs_scale<<<hs_grid(n), 256, 0, s>>>(V + (int64_t)(j + 1) * n, w, 1.0 / hn, n);
            SEM_CHECK_LAUNCH();
        }
        for (int i = k - 1; i >= 0; --i) {
            double sum = g[i];
            for (int cidx = i + 1; cidx < k; ++cidx) sum -= Hm[(size_t)i * m + cidx] * y[cidx];
            y[i] = sum / Hm[(size_t)i * m + i];
        }
        if (k > 0 && (rc = hs_maxpy(H, x, Z, n, k, y.data(), s))) return rc;
        if ((rc = true_residual(&beta))) return rc;
        if (broke) break;
        if (!isfinite(beta)) { status = SEM_ERR_BREAKDOWN; break; }
        if (beta <= target) { status = SEM_OK; break; }
        // a cycle that met its own estimate without halving the true residual
        // has reached the floor of the operators: stop there
        if (estimate_met && beta > 0.5 * beta0) break;
        ++restarts;
    }
    if (singular) {  // remove the B-weighted mean of x
        k_hs_bsum<<<HS_DOT_BLOCKS, 256, 0, s>>>(x, c->geo64, c->n * c->n * c->n, c->E, H->part);
        k_hs_dot_final<<<2, 256, 0, s>>>(H->part, HS_DOT_BLOCKS, H->dots);
        SEM_CHECK_LAUNCH();
        SEM_CUDA(cudaMemcpyAsync(H->hdots, H->dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
        k_hs_add_scalar<<<hs_grid(n), 256, 0, s>>>(x, -H->hdots[0] / H->hdots[1], n);
        SEM_CHECK_LAUNCH();
    }
    SEM_CUDA(cudaStreamSynchronize(s));
    info->status = status;
    info->iters = it;
    info->outer_iters = restarts;
    info->final_rnorm = beta;
    info->bnorm = bnorm;
    H->last = *info;
    return status;
}

extern "C" int sem_gmres_solve(sem_hsmg *H, int precond, const double *b, double *x, const sem_solve_opts *opts,
                               int restart, sem_solve_info *info, void *stream)
{
    if (!H || !b || !x || !opts || !info) return SEM_ERR_ARG;
    if (!sem_is_device_ptr(b) || !sem_is_device_ptr(x)) return SEM_ERR_ARG;
    return sem_gmres_solve_dev(H, precond, b, x, *opts, restart, info, (cudaStream_t)stream, 0);
}
