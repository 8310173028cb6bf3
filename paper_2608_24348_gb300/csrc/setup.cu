// setup.cu -- context construction: GLL tables, trilinear geometry, staging.
//
// Pre-processing of the P_N-P_N step (Sec. 1.1, Fig. 3): GLL nodes and
// weights, the derivative matrix, and per node the coordinates, J^{-1}, the
// six geometric factors G_ab = w|J| sum_c (dr_a/dx_c)(dr_b/dx_c) and the mass
// B = w|J|, all in FP64 on the device (FP32 copies for the low-precision
// operators).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

static thread_local char g_last_cuda[256];

void sem_note_cuda_error(cudaError_t e, const char *where)
{
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", where, cudaGetErrorString(e));
}

extern "C" const char *sem_last_cuda_error(void) { return g_last_cuda; }

extern "C" const char *sem_strerror(int code)
{
    switch (code) {
        case SEM_OK: return "ok";
        case SEM_ERR_ARG: return "invalid argument";
        case SEM_ERR_CUDA: return "CUDA runtime error";
        case SEM_ERR_NOMEM: return "out of memory";
        case SEM_ERR_BAD_MESH: return "non-positive Jacobian determinant";
        case SEM_ERR_NOT_CONVERGED: return "solver did not converge";
        case SEM_ERR_BREAKDOWN: return "solver breakdown";
        case SEM_ERR_TIMEOUT: return "device-side wait timed out";
        case SEM_ERR_TOO_LARGE: return "problem exceeds the fixed scratch size";
        default: return "unknown error";
    }
}

// ---------------------------------------------------------------------------
// 1-D tables (host, FP64)
// ---------------------------------------------------------------------------

// P_m(x) for m = n-1, n, n+1 by the Bonnet recurrence.
static void legendre3(int N, double x, double *pm1, double *p, double *pp1)
{
    double a = 1.0, b = x;  // P_0, P_1
    if (N == 0) { *pm1 = 0; *p = 1; *pp1 = x; return; }
    double prev = a, cur = b;
    for (int k = 1; k < N; ++k) {
        double nxt = ((2 * k + 1) * x * cur - k * prev) / (k + 1);
        prev = cur;
        cur = nxt;
    }
    *pm1 = prev;
    *p = cur;
    *pp1 = ((2 * N + 1) * x * cur - N * prev) / (N + 1);
}

// GLL nodes are the roots of q = P_{N+1} - P_{N-1} (which is proportional to
// (1 - x^2) P_N'); q' = (2N+1) P_N.  Newton from Chebyshev-Lobatto points.
static void gll_table(int N, double *xi, double *w)
{
    for (int i = 0; i <= N; ++i) {
        double x = -cos(M_PI * i / N);
        if (i > 0 && i < N) {
            for (int it = 0; it < 60; ++it) {
                double pm1, p, pp1;
                legendre3(N, x, &pm1, &p, &pp1);
                double dx = (pp1 - pm1) / ((2 * N + 1) * p);
                x -= dx;
                if (fabs(dx) < 1e-17) break;
            }
        }
        xi[i] = x;
    }
    for (int i = 0; i < (N + 1) / 2; ++i) {  // exact symmetry
        double s = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -s;
        xi[N - i] = s;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int i = 0; i <= N; ++i) {
        double pm1, p, pp1;
        legendre3(N, xi[i], &pm1, &p, &pp1);
        w[i] = 2.0 / (N * (N + 1.0) * p * p);
    }
}

// D_ij = l_j'(xi_i) from barycentric weights lam_j = 1 / prod_{k!=j}(xi_j - xi_k):
// D_ij = (lam_j / lam_i) / (xi_i - xi_j), diagonal = -(row sum).
static void deriv_table(int N, const double *xi, double *D)
{
    int n = N + 1;
    double lam[SEM_NPMAX];
    for (int j = 0; j < n; ++j) {
        double pr = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) pr *= (xi[j] - xi[k]);
        lam[j] = 1.0 / pr;
    }
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double v = (lam[j] / lam[i]) / (xi[i] - xi[j]);
            D[i * n + j] = v;
            s += v;
        }
        D[i * n + i] = -s;
    }
}

// ---------------------------------------------------------------------------
// Geometry kernel: one thread per local node
// ---------------------------------------------------------------------------

struct GeoArgs {
    int N, n, nelx, nely, nelz;
    int64_t nL;
    const double *vert;
    const double *xi, *w;
    double *geo64;
    float *geo32;
    double *xyz;      // may be null
    double *jinv64;   // may be null
    float *jinv32;    // may be null
    int *bad;
};

__global__ void k_geometry(GeoArgs a)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= a.nL) return;
    const int n = a.n, n3 = n * n * n;
    int64_t e = p / n3;
    int l = (int)(p - e * n3);
    int i = l % n, j = (l / n) % n, k = l / (n * n);
    int ex = (int)(e % a.nelx), ey = (int)((e / a.nelx) % a.nely), ez = (int)(e / ((int64_t)a.nelx * a.nely));
    // trilinear map x = c0 + c1 r + c2 s + c3 t + c4 rs + c5 rt + c6 st + c7 rst
    double c[8][3];
    for (int m = 0; m < 8; ++m) c[m][0] = c[m][1] = c[m][2] = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                int64_t vi = ((int64_t)(ez + cz) * (a.nely + 1) + (ey + cy)) * (a.nelx + 1) + (ex + cx);
                double sx = cx ? 1.0 : -1.0, sy = cy ? 1.0 : -1.0, sz = cz ? 1.0 : -1.0;
                double sg[8] = {1.0, sx, sy, sz, sx * sy, sx * sz, sy * sz, sx * sy * sz};
                for (int d = 0; d < 3; ++d) {
                    double v = 0.125 * a.vert[vi * 3 + d];
                    for (int m = 0; m < 8; ++m) c[m][d] += sg[m] * v;
                }
            }
    const double r = a.xi[i], s = a.xi[j], t = a.xi[k];
    double X[3], J[3][3];  // J[d][a] = dx_d / dr_a
    for (int d = 0; d < 3; ++d) {
        X[d] = c[0][d] + c[1][d] * r + c[2][d] * s + c[3][d] * t + c[4][d] * r * s + c[5][d] * r * t +
               c[6][d] * s * t + c[7][d] * r * s * t;
        J[d][0] = c[1][d] + c[4][d] * s + c[5][d] * t + c[7][d] * s * t;
        J[d][1] = c[2][d] + c[4][d] * r + c[6][d] * t + c[7][d] * r * t;
        J[d][2] = c[3][d] + c[5][d] * r + c[6][d] * s + c[7][d] * r * s;
    }
    // adjugate: adj[a][d] = cofactor(d, a)
    double adj[3][3];
    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
    if (!(det > 0.0)) atomicOr(a.bad, 1);
    const double inv_det = 1.0 / det;
    double R[3][3];  // R[a][d] = dr_a / dx_d
    for (int x = 0; x < 3; ++x)
        for (int d = 0; d < 3; ++d) R[x][d] = adj[x][d] * inv_det;
    const double bm = a.w[i] * a.w[j] * a.w[k] * det;
    double g[7];
    g[0] = bm * (R[0][0] * R[0][0] + R[0][1] * R[0][1] + R[0][2] * R[0][2]);
    g[1] = bm * (R[1][0] * R[1][0] + R[1][1] * R[1][1] + R[1][2] * R[1][2]);
    g[2] = bm * (R[2][0] * R[2][0] + R[2][1] * R[2][1] + R[2][2] * R[2][2]);
    g[3] = bm * (R[0][0] * R[1][0] + R[0][1] * R[1][1] + R[0][2] * R[1][2]);
    g[4] = bm * (R[0][0] * R[2][0] + R[0][1] * R[2][1] + R[0][2] * R[2][2]);
    g[5] = bm * (R[1][0] * R[2][0] + R[1][1] * R[2][1] + R[1][2] * R[2][2]);
    g[6] = bm;
    double *G64 = a.geo64 + e * 7 * n3 + l;
    float *G32 = a.geo32 + e * 7 * n3 + l;
    for (int m = 0; m < 7; ++m) {
        G64[(int64_t)m * n3] = g[m];
        G32[(int64_t)m * n3] = (float)g[m];
    }
    if (a.xyz)
        for (int d = 0; d < 3; ++d) a.xyz[d * a.nL + p] = X[d];
    if (a.jinv64) {
        for (int x = 0; x < 3; ++x)
            for (int d = 0; d < 3; ++d) {
                a.jinv64[(e * 9 + x * 3 + d) * n3 + l] = R[x][d];
                a.jinv32[(e * 9 + x * 3 + d) * n3 + l] = (float)R[x][d];
            }
    }
}

// Deterministic sum of the mass: one partial per block, then a single block.
__global__ void k_sum_B_partial(const double *geo64, int64_t E, int n3, double *part)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x)
        for (int l = threadIdx.x; l < n3; l += blockDim.x) s += geo64[(e * 7 + 6) * n3 + l];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_serial(const double *part, int np, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < np; ++b) s += part[b];
        *out = s;
    }
}

__global__ void k_uniform_vertices(double *vert, int nelx, int nely, int nelz, double Lx, double Ly,
                                   double Lz)
{
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nv = (int64_t)(nelx + 1) * (nely + 1) * (nelz + 1);
    if (v >= nv) return;
    int I = (int)(v % (nelx + 1)), J = (int)((v / (nelx + 1)) % (nely + 1)),
        K = (int)(v / ((int64_t)(nelx + 1) * (nely + 1)));
    vert[v * 3 + 0] = Lx * I / nelx;
    vert[v * 3 + 1] = Ly * J / nely;
    vert[v * 3 + 2] = Lz * K / nelz;
}

// ---------------------------------------------------------------------------
// Geometry pass (used by setup and, with J^{-1}, by the stepper)
// ---------------------------------------------------------------------------

int sem_run_geometry(sem_ctx *c, double *xyz, bool with_jinv, cudaStream_t s)
{
    int *bad = nullptr;
    SEM_CUDA(cudaMallocAsync(&bad, sizeof(int), s));
    SEM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    GeoArgs a;
    a.N = c->N; a.n = c->n; a.nelx = c->nelx; a.nely = c->nely; a.nelz = c->nelz;
    a.nL = c->nL;
    a.vert = c->vert;
    a.xi = c->tab64;
    a.w = c->tab64 + c->n;
    a.geo64 = c->geo64;
    a.geo32 = c->geo32;
    a.xyz = xyz;
    a.jinv64 = with_jinv ? c->jinv64 : nullptr;
    a.jinv32 = with_jinv ? c->jinv32 : nullptr;
    a.bad = bad;
    k_geometry<<<(unsigned)sem_ceil_div(c->nL, 256), 256, 0, s>>>(a);
    SEM_CHECK_LAUNCH();
    int hbad = 0;
    SEM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaFreeAsync(bad, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    return hbad ? SEM_ERR_BAD_MESH : SEM_OK;
}

int sem_alloc_ws(sem_ctx *c, int slot)
{
    sem_ws &w = c->ws[slot];
    size_t n64 = (size_t)c->nL * sizeof(double), n32 = (size_t)c->nL * sizeof(float);
    double **d64[] = {&w.r, &w.p, &w.w, &w.minv, &w.b};
    float **d32[] = {&w.r32, &w.p32, &w.w32, &w.d32, &w.minv32};
    for (auto pp : d64)
        if (cudaMalloc(pp, n64) != cudaSuccess) return SEM_ERR_NOMEM;
    for (auto pp : d32)
        if (cudaMalloc(pp, n32) != cudaSuccess) return SEM_ERR_NOMEM;
    return SEM_OK;
}

static void free_ws(sem_ws &w)
{
    void *ps[] = {w.r, w.p, w.w, w.minv, w.b, w.r32, w.p32, w.w32, w.d32, w.minv32};
    for (void *p : ps)
        if (p) cudaFree(p);
    memset(&w, 0, sizeof(w));
}

void sem_pipe_destroy(void *pipe);  // ops.cu

extern "C" void sem_destroy(sem_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    sem_pipe_destroy(c->pipe);
    void *ps[] = {c->tab64, c->tab32, c->geo64, c->geo32, c->geodf, c->tabdf, c->tabdfeo, c->vert, c->jinv64, c->jinv32, c->err_dev,
                  c->solve_dev, c->partials, c->stage[0], c->stage[1]};
    for (void *p : ps)
        if (p) cudaFree(p);
    free(c->bfp_tabs);
    if (c->solve_host) cudaFreeHost(c->solve_host);
    for (int s = 0; s < 8; ++s) free_ws(c->ws[s]);
    free(c);
}

int sem_solve_state_bytes();             // pcg.cu
int sem_make_geo_df(sem_ctx *c);         // ax_df.cu
int sem_solve_upload_tables(const sem_ctx *c);  // pcg.cu
size_t sem_partials_bytes(int num_sms);  // pcg.cu

extern "C" int sem_setup(int N, int nelx, int nely, int nelz, const double extents[3],
                         const int periodic[3], const double *vertices, sem_ctx **out)
{
    if (!out) return SEM_ERR_ARG;
    *out = nullptr;
    if (N < 1 || N > SEM_NMAX || nelx < 1 || nely < 1 || nelz < 1 || !periodic) return SEM_ERR_ARG;
    if (!vertices && !extents) return SEM_ERR_ARG;
    if ((int64_t)nelx * N > (1 << 30) || (int64_t)nely * N > (1 << 30) || (int64_t)nelz * N > (1 << 30))
        return SEM_ERR_ARG;
    if (((int64_t)nely * N + 1) * ((int64_t)nelz * N + 1) >= ((int64_t)1 << 31) - 8) return SEM_ERR_ARG;
    sem_ctx *c = (sem_ctx *)calloc(1, sizeof(sem_ctx));
    if (!c) return SEM_ERR_NOMEM;
    c->N = N;
    c->n = N + 1;
    c->nelx = nelx; c->nely = nely; c->nelz = nelz;
    for (int d = 0; d < 3; ++d) c->periodic[d] = periodic[d] ? 1 : 0;
    c->E = (int64_t)nelx * nely * nelz;
    c->nL = c->E * c->n * c->n * c->n;
    c->ngx = nelx * N + (c->periodic[0] ? 0 : 1);
    c->ngy = nely * N + (c->periodic[1] ? 0 : 1);
    c->ngz = nelz * N + (c->periodic[2] ? 0 : 1);
    c->nG = (int64_t)c->ngx * c->ngy * c->ngz;
    int rc = SEM_OK;
    cudaStream_t s = 0;
#define SETUP_TRY(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            sem_note_cuda_error(e_, #call);               \
            sem_destroy(c);                               \
            return e_ == cudaErrorMemoryAllocation ? SEM_ERR_NOMEM : SEM_ERR_CUDA; \
        }                                                 \
    } while (0)
    SETUP_TRY(cudaGetDevice(&c->device));
    SETUP_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    gll_table(N, c->hxi, c->hw);
    deriv_table(N, c->hxi, c->hD);
    const int n = c->n;
    double h64[2 * SEM_NPMAX + SEM_NPMAX * SEM_NPMAX];
    float h32[2 * SEM_NPMAX + SEM_NPMAX * SEM_NPMAX];
    int ntab = 2 * n + n * n;
    for (int i = 0; i < n; ++i) { h64[i] = c->hxi[i]; h64[n + i] = c->hw[i]; }
    for (int i = 0; i < n * n; ++i) h64[2 * n + i] = c->hD[i];
    for (int i = 0; i < ntab; ++i) h32[i] = (float)h64[i];
    SETUP_TRY(cudaMalloc(&c->tab64, sizeof(double) * ntab));
    SETUP_TRY(cudaMalloc(&c->tab32, sizeof(float) * ntab));
    SETUP_TRY(cudaMemcpy(c->tab64, h64, sizeof(double) * ntab, cudaMemcpyHostToDevice));
    SETUP_TRY(cudaMemcpy(c->tab32, h32, sizeof(float) * ntab, cudaMemcpyHostToDevice));
    size_t nv = (size_t)(nelx + 1) * (nely + 1) * (nelz + 1) * 3;
    SETUP_TRY(cudaMalloc(&c->vert, sizeof(double) * nv));
    if (vertices) {
        SETUP_TRY(cudaMemcpy(c->vert, vertices, sizeof(double) * nv, cudaMemcpyHostToDevice));
        for (int d = 0; d < 3; ++d) c->L[d] = extents ? extents[d] : 0.0;
    } else {
        for (int d = 0; d < 3; ++d) {
            if (!(extents[d] > 0)) { sem_destroy(c); return SEM_ERR_ARG; }
            c->L[d] = extents[d];
        }
        int64_t nvp = (int64_t)nv / 3;
        k_uniform_vertices<<<(unsigned)sem_ceil_div(nvp, 256), 256>>>(c->vert, nelx, nely, nelz,
                                                                        c->L[0], c->L[1], c->L[2]);
    }
    SETUP_TRY(cudaMalloc(&c->geo64, sizeof(double) * 7 * c->nL));
    SETUP_TRY(cudaMalloc(&c->geo32, sizeof(float) * 7 * c->nL));
    rc = sem_run_geometry(c, nullptr, false, s);
    if (rc != SEM_OK) { sem_destroy(c); return rc; }
    rc = sem_make_geo_df(c);
    if (rc != SEM_OK) { sem_destroy(c); return rc; }
    rc = sem_solve_upload_tables(c);
    if (rc != SEM_OK) { sem_destroy(c); return rc; }
    // volume = sum of B
    {
        double *part = nullptr;
        int nb = 1024;
        SETUP_TRY(cudaMalloc(&part, sizeof(double) * (nb + 1)));
        k_sum_B_partial<<<nb, 256>>>(c->geo64, c->E, n * n * n, part);
        k_sum_serial<<<1, 32>>>(part, nb, part + nb);
        SETUP_TRY(cudaMemcpy(&c->volume, part + nb, sizeof(double), cudaMemcpyDeviceToHost));
        cudaFree(part);
    }
    // solver workspace slot 0 and solve state
    c->nws = 1;
    rc = sem_alloc_ws(c, 0);
    if (rc != SEM_OK) { sem_destroy(c); return rc; }
    SETUP_TRY(cudaMalloc(&c->solve_dev, sem_solve_state_bytes()));
    SETUP_TRY(cudaMemset(c->solve_dev, 0, sem_solve_state_bytes()));
    SETUP_TRY(cudaMallocHost(&c->solve_host, sem_solve_state_bytes()));
    SETUP_TRY(cudaMalloc(&c->partials, sem_partials_bytes(c->num_sms)));
    SETUP_TRY(cudaMalloc(&c->err_dev, sizeof(int)));
    SETUP_TRY(cudaMemset(c->err_dev, 0, sizeof(int)));
    memset(c->solve_host, 0, sem_solve_state_bytes());
    SETUP_TRY(cudaDeviceSynchronize());
#undef SETUP_TRY
    *out = c;
    return SEM_OK;
}

extern "C" int sem_device_status(sem_ctx *c)
{
    if (!c) return SEM_ERR_ARG;
    int h = 0;
    SEM_CUDA(cudaMemcpy(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    SEM_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
    return h;
}

extern "C" int sem_get_info(const sem_ctx *c, sem_ctx_info *info)
{
    if (!c || !info) return SEM_ERR_ARG;
    info->N = c->N;
    info->nelx = c->nelx; info->nely = c->nely; info->nelz = c->nelz;
    for (int d = 0; d < 3; ++d) info->periodic[d] = c->periodic[d];
    info->E = c->E;
    info->nL = c->nL;
    info->nG = c->nG;
    info->volume = c->volume;
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// Pointer staging for host buffers
// ---------------------------------------------------------------------------

int sem_is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int sem_ensure_stage(sem_ctx *c, size_t bytes)
{
    if (bytes <= c->stage_bytes) return SEM_OK;
    for (int k = 0; k < 2; ++k) {
        if (c->stage[k]) cudaFree(c->stage[k]);
        c->stage[k] = nullptr;
    }
    c->stage_bytes = 0;
    for (int k = 0; k < 2; ++k)
        if (cudaMalloc(&c->stage[k], bytes) != cudaSuccess) return SEM_ERR_NOMEM;
    c->stage_bytes = bytes;
    return SEM_OK;
}

int sem_stage_in(sem_ctx *c, const void *p, size_t bytes, int slot, cudaStream_t s, const void **dev,
                 int *is_host)
{
    if (sem_is_device_ptr(p)) {
        *dev = p;
        *is_host = 0;
        return SEM_OK;
    }
    int rc = sem_ensure_stage(c, bytes);
    if (rc) return rc;
    SEM_CUDA(cudaMemcpyAsync(c->stage[slot], p, bytes, cudaMemcpyHostToDevice, s));
    *dev = c->stage[slot];
    *is_host = 1;
    return SEM_OK;
}

int sem_stage_out_ptr(sem_ctx *c, void *p, size_t bytes, int slot, void **dev, int *is_host)
{
    if (sem_is_device_ptr(p)) {
        *dev = p;
        *is_host = 0;
        return SEM_OK;
    }
    int rc = sem_ensure_stage(c, bytes);
    if (rc) return rc;
    *dev = c->stage[slot];
    *is_host = 1;
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// Exports of setup data
// ---------------------------------------------------------------------------

__global__ void k_copy_geo(const double *geo64, double *out, int64_t E, int n3)
{
    // out: 7 E-vectors; geo64: [E][7][n3]
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nL = E * n3;
    if (t >= 7 * nL) return;
    int m = (int)(t / nL);
    int64_t p = t - m * nL;
    int64_t e = p / n3;
    int l = (int)(p - e * n3);
    out[t] = geo64[(e * 7 + m) * n3 + l];
}

extern "C" int sem_geom(sem_ctx *c, double *out, void *stream)
{
    if (!c || !out) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    void *dev;
    int host;
    size_t bytes = sizeof(double) * 7 * c->nL;
    int rc = sem_stage_out_ptr(c, out, bytes, 1, &dev, &host);
    if (rc) return rc;
    if (host && bytes > c->stage_bytes) return SEM_ERR_ARG;
    k_copy_geo<<<(unsigned)sem_ceil_div(7 * c->nL, 256), 256, 0, s>>>(c->geo64, (double *)dev, c->E,
                                                                       c->n * c->n * c->n);
    SEM_CHECK_LAUNCH();
    if (host) {
        SEM_CUDA(cudaMemcpyAsync(out, dev, bytes, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
    }
    return SEM_OK;
}

extern "C" int sem_coords(sem_ctx *c, double *xyz, void *stream)
{
    if (!c || !xyz) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    void *dev;
    int host;
    size_t bytes = sizeof(double) * 3 * c->nL;
    int rc = sem_stage_out_ptr(c, xyz, bytes, 1, &dev, &host);
    if (rc) return rc;
    SEM_CUDA(cudaStreamSynchronize(s));
    rc = sem_run_geometry(c, (double *)dev, false, s);
    if (rc) return rc;
    if (host) {
        SEM_CUDA(cudaMemcpyAsync(xyz, dev, bytes, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
    }
    return SEM_OK;
}
