// ops.cu -- stand-alone operator entry points: sem_ax, sem_dssum, sem_jacobi.
#include "common.cuh"
#include "gs.cuh"

int sem_ax_tc(sem_ctx *c, const float *u, float *w, double h1, double h2, int fp16,
              cudaStream_t s);  // ax_tc.cu
int sem_launch_ax_f64(const sem_ctx *c, const double *u, double *w, double h1, double h2,
                      cudaStream_t s);  // ax_f64.cu
int sem_launch_ax_f32_variant(const sem_ctx *c, int variant, const float *u, float *w, float h1,
                              float h2, cudaStream_t s);  // ax_f32.cu
int sem_launch_ax_df(const sem_ctx *c, const double *u, double *w, double h1, double h2,
                     cudaStream_t s);   // ax_df.cu

// ---------------------------------------------------------------------------
// Per-order kernel choice (the tile shape of the stand-alone operator)
// ---------------------------------------------------------------------------

#define SEM_NVARIANT 3
static int g_variant[SEM_NMAX + 1][5];  // 0 = not set -> built-in default
static int g_variant_set[SEM_NMAX + 1][5];

// Built-in defaults from measurements on GB300: staged 128 x 3 for N = 7 and
// 9, staged 256 x 2 for N = 3 and 5, direct loads otherwise.
static int default_variant(int N, sem_dtype dt)
{
    if (dt != SEM_F32) return 0;
    if (N == 7 || N == 9) return 2;
    if (N == 3 || N == 5) return 1;
    return 0;
}

int sem_ax_variant(int N, sem_dtype dt)
{
    if (N < 1 || N > SEM_NMAX || dt < SEM_F64 || dt > SEM_F64_NATIVE) return 0;
    return g_variant_set[N][dt] ? g_variant[N][dt] : default_variant(N, dt);
}

extern "C" int sem_set_ax_variant(int N, sem_dtype dt, int variant)
{
    if (N < 1 || N > SEM_NMAX || dt < SEM_F64 || dt > SEM_F64_NATIVE) return SEM_ERR_ARG;
    if (variant < 0 || variant >= SEM_NVARIANT || (dt != SEM_F32 && variant != 0)) return SEM_ERR_ARG;
    g_variant[N][dt] = variant;
    g_variant_set[N][dt] = 1;
    return SEM_OK;
}

GsDesc sem_gs_desc(const sem_ctx *c)
{
    GsDesc d;
    d.N = c->N; d.n = c->n;
    d.nelx = c->nelx; d.nely = c->nely; d.nelz = c->nelz;
    d.ngx = c->ngx; d.ngy = c->ngy; d.ngz = c->ngz;
    d.px = c->periodic[0]; d.py = c->periodic[1]; d.pz = c->periodic[2];
    d.nG = c->nG;
    return d;
}

int sem_ax_variant(int N, sem_dtype dt);

// Device-pointer form (used by the stepper as well).
int sem_ax_dev(sem_ctx *c, const void *u, void *w, double h1, double h2, sem_dtype dt,
               cudaStream_t s)
{
    if (c->E == 0) return SEM_OK;
    if (dt == SEM_F64) {
        return sem_launch_ax_df(c, (const double *)u, (double *)w, h1, h2, s);
    } else if (dt == SEM_F64_NATIVE) {
        return sem_launch_ax_f64(c, (const double *)u, (double *)w, h1, h2, s);
    } else if (dt == SEM_F32) {
        return sem_launch_ax_f32_variant(c, sem_ax_variant(c->N, SEM_F32), (const float *)u, (float *)w,
                                         (float)h1, (float)h2, s);
    } else if (dt == SEM_BF16_TC || dt == SEM_F16_TC) {
        return sem_ax_tc(c, (const float *)u, (float *)w, h1, h2, dt == SEM_F16_TC, s);
    }
    return SEM_ERR_ARG;
}

extern "C" int sem_ax(sem_ctx *c, const void *u, void *w, double h1, double h2, sem_dtype dt,
                      void *stream)
{
    if (!c || !u || !w) return SEM_ERR_ARG;
    if (dt < SEM_F64 || dt > SEM_F64_NATIVE) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool f64 = dt == SEM_F64 || dt == SEM_F64_NATIVE;
    size_t bytes = (size_t)c->nL * (f64 ? sizeof(double) : sizeof(float));
    const void *ud;
    void *wd;
    int uh, wh;
    int rc = sem_stage_in(c, u, bytes, 0, s, &ud, &uh);
    if (rc) return rc;
    rc = sem_stage_out_ptr(c, w, bytes, 1, &wd, &wh);
    if (rc) return rc;
    rc = sem_ax_dev(c, ud, wd, h1, h2, dt, s);
    if (rc) return rc;
    if (wh) {
        SEM_CUDA(cudaMemcpyAsync(w, wd, bytes, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
    } else if (uh) {
        SEM_CUDA(cudaStreamSynchronize(s));
    }
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// dssum: one thread per unique node, owner computes, no atomics
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_dssum(T *__restrict__ u, GsDesc d)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= d.nG) return;
    int64_t idx[8];
    int m = gs_copies(d, g, idx);
    if (m == 1) return;
    T s = T(0);
    for (int t = 0; t < m; ++t) s += u[idx[t]];
    for (int t = 0; t < m; ++t) u[idx[t]] = s;
}

int sem_dssum_dev(sem_ctx *c, void *u, sem_dtype dt, cudaStream_t s)
{
    if (c->nG == 0) return SEM_OK;
    GsDesc d = sem_gs_desc(c);
    unsigned grid = (unsigned)sem_ceil_div(c->nG, 256);
    if (dt == SEM_F64)
        k_dssum<double><<<grid, 256, 0, s>>>((double *)u, d);
    else
        k_dssum<float><<<grid, 256, 0, s>>>((float *)u, d);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

extern "C" int sem_dssum(sem_ctx *c, void *u, sem_dtype dt, void *stream)
{
    if (!c || !u) return SEM_ERR_ARG;
    if (dt < SEM_F64 || dt > SEM_F16_TC) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)c->nL * (dt == SEM_F64 ? sizeof(double) : sizeof(float));
    const void *ud;
    int uh;
    int rc = sem_stage_in(c, u, bytes, 0, s, &ud, &uh);
    if (rc) return rc;
    rc = sem_dssum_dev(c, (void *)ud, dt, s);
    if (rc) return rc;
    if (uh) {
        SEM_CUDA(cudaMemcpyAsync(u, ud, bytes, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
    }
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// Jacobi diagonal
// ---------------------------------------------------------------------------

// Local diagonal of the element operator (cross terms included).
__global__ void k_jacobi_local(const double *__restrict__ geo, const double *__restrict__ D,
                               double h1, double h2, int n, int64_t nL, double *__restrict__ out)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nL) return;
    const int n3 = n * n * n;
    int64_t e = p / n3;
    int l = (int)(p - e * n3);
    int i = l % n, j = (l / n) % n, k = l / (n * n);
    const double *g = geo + e * 7 * n3;
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
        double a = D[m * n + i], b = D[m * n + j], c = D[m * n + k];
        s += a * a * g[0 * n3 + (k * n + j) * n + m];
        s += b * b * g[1 * n3 + (k * n + m) * n + i];
        s += c * c * g[2 * n3 + (m * n + j) * n + i];
    }
    const double di = D[i * n + i], dj = D[j * n + j], dk = D[k * n + k];
    s += 2.0 * (di * dj * g[3 * n3 + l] + di * dk * g[4 * n3 + l] + dj * dk * g[5 * n3 + l]);
    out[p] = h1 * s + h2 * g[6 * n3 + l];
}

// dssum fused with the reciprocal: every copy receives 1 / (sum of copies).
__global__ void k_dssum_recip(double *__restrict__ u, float *__restrict__ u32, GsDesc d)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= d.nG) return;
    int64_t idx[8];
    int m = gs_copies(d, g, idx);
    double s = 0.0;
    for (int t = 0; t < m; ++t) s += u[idx[t]];
    double r = 1.0 / s;
    for (int t = 0; t < m; ++t) {
        u[idx[t]] = r;
        if (u32) u32[idx[t]] = (float)r;
    }
}

int sem_jacobi_dev(sem_ctx *c, double h1, double h2, double *minv, float *minv32, cudaStream_t s)
{
    if (c->nL == 0) return SEM_OK;
    k_jacobi_local<<<(unsigned)sem_ceil_div(c->nL, 256), 256, 0, s>>>(c->geo64, c->tab64 + 2 * c->n,
                                                                       h1, h2, c->n, c->nL, minv);
    SEM_CHECK_LAUNCH();
    GsDesc d = sem_gs_desc(c);
    k_dssum_recip<<<(unsigned)sem_ceil_div(c->nG, 256), 256, 0, s>>>(minv, minv32, d);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

extern "C" int sem_jacobi(sem_ctx *c, double h1, double h2, double *minv, void *stream)
{
    if (!c || !minv) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    void *dev;
    int host;
    size_t bytes = sizeof(double) * c->nL;
    int rc = sem_stage_out_ptr(c, minv, bytes, 1, &dev, &host);
    if (rc) return rc;
    rc = sem_jacobi_dev(c, h1, h2, (double *)dev, nullptr, s);
    if (rc) return rc;
    if (host) {
        SEM_CUDA(cudaMemcpyAsync(minv, dev, bytes, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
    }
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the stand-alone operator's tile shape
// ---------------------------------------------------------------------------

extern "C" int sem_tune_ax(sem_ctx *c, sem_dtype dt, int reps, double *ms, int *best)
{
    if (!c || !best || dt < SEM_F64 || dt > SEM_F64_NATIVE) return SEM_ERR_ARG;
    if (reps < 1) reps = 5;
    const int nvar = dt == SEM_F32 ? SEM_NVARIANT : 1;
    // the solver workspace of slot 0 serves as input and output (its contents
    // are scratch between solves); u = r32, w = w32
    const float *u = c->ws[0].r32;
    float *w = c->ws[0].w32;
    cudaStream_t s = 0;
    cudaEvent_t e0, e1;
    SEM_CUDA(cudaEventCreate(&e0));
    SEM_CUDA(cudaEventCreate(&e1));
    SEM_CUDA(cudaMemsetAsync((void *)u, 0, sizeof(float) * c->nL, s));
    double best_ms = 1e300;
    int bi = 0;
    for (int v = 0; v < nvar; ++v) {
        double t = 1e300;
        int rc = SEM_OK;
        if (dt == SEM_F32) {
            rc = sem_launch_ax_f32_variant(c, v, u, w, 1.0f, 1.0f, s);  // warm-up
            if (rc == SEM_OK) {
                SEM_CUDA(cudaEventRecord(e0, s));
                for (int k = 0; k < reps && rc == SEM_OK; ++k)
                    rc = sem_launch_ax_f32_variant(c, v, u, w, 1.0f, 1.0f, s);
                SEM_CUDA(cudaEventRecord(e1, s));
                SEM_CUDA(cudaEventSynchronize(e1));
                float f = 0.f;
                SEM_CUDA(cudaEventElapsedTime(&f, e0, e1));
                t = f / reps;
            }
        } else {
            t = 0.0;
        }
        if (ms) ms[v] = rc == SEM_OK ? t : -1.0;
        if (rc == SEM_OK && t < best_ms) {
            best_ms = t;
            bi = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best = bi;
    return sem_set_ax_variant(c->N, dt, bi);
}
