// ops.cu -- stand-alone operator entry points: sem_ax, sem_dssum, sem_jacobi.
#include <stdlib.h>

#include "common.cuh"
#include "gs.cuh"

int sem_ax_tc(sem_ctx *c, const float *u, float *w, double h1, double h2, int fp16,
              cudaStream_t s);  // ax_tc.cu
int sem_ax_tc_split(sem_ctx *c, const float *u, float *w, double h1, double h2, int fp16,
                    cudaStream_t s);  // ax_tc.cu
int sem_launch_ax_f64_v(const sem_ctx *c, const double *u, double *w, double h1, double h2, int fold,
                        cudaStream_t s);
int sem_launch_ax_f64(const sem_ctx *c, const double *u, double *w, double h1, double h2,
                      cudaStream_t s);  // ax_f64.cu
int sem_launch_ax_f32_variant(const sem_ctx *c, int variant, const float *u, float *w, float h1,
                              float h2, cudaStream_t s);  // ax_f32.cu
int sem_launch_ax_df(const sem_ctx *c, const double *u, double *w, double h1, double h2,
                     cudaStream_t s);   // ax_df.cu

// ---------------------------------------------------------------------------
// Per-order kernel choice (the tile shape of the stand-alone operator)
// ---------------------------------------------------------------------------

// Candidates per dtype: SEM_F32 three tile shapes; SEM_F64 three shapes of the
// float-pair folded kernel and the block-floating-point kernel with scalar (3)
// and paired (4) FP32 instructions, each also with u staged by bulk copies (5, 6),
// and the staged scalar form with half (7) and one (8) element per block, the
// latter also with register budgets for 20 (9) and 24 (10) warps per SM.
#define SEM_NVARIANT 11
static_assert(SEM_NVARIANT <= SEM_TUNE_MAX, "tuner output array");
static int sem_nvariant(sem_dtype dt) { return dt == SEM_F64 ? 11 : dt == SEM_F32 ? 3 : dt == SEM_F64_NATIVE ? 2 : 1; }
static int g_variant[SEM_NMAX + 1][5];  // 0 = not set -> built-in default
static int g_variant_set[SEM_NMAX + 1][5];

// Built-in defaults from measurements on GB300.  FP32: staged 128 x 3 for
// N = 7 and 9, staged 256 x 2 for N = 3 and 5, direct loads otherwise.
// FP64-accurate: the block-floating-point kernel with u staged, one element
// per block (0.27 ms against 0.43 ms for the float-pair folded kernel at 32^3,
// N = 7), for odd N <= 11 (even N+1 <= 12); the float-pair kernels otherwise.
static int default_variant(int N, sem_dtype dt)
{
    if (dt == SEM_F64) return (N % 2 == 1 && N <= 11) ? 8 : 0;
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
    if (variant == -1) {  // back to the built-in default
        g_variant_set[N][dt] = 0;
        return SEM_OK;
    }
    if (variant < 0 || variant >= sem_nvariant(dt)) return SEM_ERR_ARG;
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

// Device-pointer form (used by the stepper as well).
int sem_ax_dev(sem_ctx *c, const void *u, void *w, double h1, double h2, sem_dtype dt,
               cudaStream_t s)
{
    if (c->E == 0) return SEM_OK;
    if (dt == SEM_F64) {
        return sem_launch_ax_df(c, (const double *)u, (double *)w, h1, h2, s);
    } else if (dt == SEM_F64_NATIVE) {
        return sem_launch_ax_f64_v(c, (const double *)u, (double *)w, h1, h2,
                                   sem_ax_variant(c->N, SEM_F64_NATIVE) == 0, s);
    } else if (dt == SEM_F32) {
        return sem_launch_ax_f32_variant(c, sem_ax_variant(c->N, SEM_F32), (const float *)u, (float *)w,
                                         (float)h1, (float)h2, s);
    } else if (dt == SEM_BF16_TC || dt == SEM_F16_TC) {
        return sem_ax_tc(c, (const float *)u, (float *)w, h1, h2, dt == SEM_F16_TC, s);
    } else if (dt == SEM_F16X2_TC || dt == SEM_BF16X3_TC) {
        return sem_ax_tc_split(c, (const float *)u, (float *)w, h1, h2, dt == SEM_F16X2_TC, s);
    }
    return SEM_ERR_ARG;
}

// ---------------------------------------------------------------------------
// Host buffers: the operator in element chunks on three streams, so that the
// copy of chunk k+1 to the device, the operator on chunk k and the copy of
// chunk k-1 back to the host overlap (the host link carries both directions
// at once).  A chunk is a contiguous element range; its geometry is the same
// range of the element-blocked factors.
// ---------------------------------------------------------------------------

#ifndef SEM_PIPE_CHUNKS
#define SEM_PIPE_CHUNKS 8
#endif

struct AxPipe {
    cudaStream_t in, out;
    cudaEvent_t start, done, ev_in[SEM_PIPE_CHUNKS], ev_cmp[SEM_PIPE_CHUNKS];
};

void sem_pipe_destroy(void *pipe)
{
    AxPipe *P = (AxPipe *)pipe;
    if (!P) return;
    // handles that were never created are null (the struct is zero-initialised)
    if (P->in) cudaStreamDestroy(P->in);
    if (P->out) cudaStreamDestroy(P->out);
    if (P->start) cudaEventDestroy(P->start);
    if (P->done) cudaEventDestroy(P->done);
    for (int k = 0; k < SEM_PIPE_CHUNKS; ++k) {
        if (P->ev_in[k]) cudaEventDestroy(P->ev_in[k]);
        if (P->ev_cmp[k]) cudaEventDestroy(P->ev_cmp[k]);
    }
    free(P);
}

static AxPipe *ax_pipe(sem_ctx *c)
{
    if (c->pipe) return (AxPipe *)c->pipe;
    AxPipe *P = (AxPipe *)calloc(1, sizeof(AxPipe));
    if (!P) return nullptr;
    bool ok = cudaStreamCreateWithFlags(&P->in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&P->out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&P->start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < SEM_PIPE_CHUNKS; ++k)
        ok = cudaEventCreateWithFlags(&P->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&P->ev_cmp[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        sem_pipe_destroy(P);
        return nullptr;
    }
    c->pipe = P;
    return P;
}

int sem_ensure_stage(sem_ctx *c, size_t bytes);  // setup.cu

static int ax_host(sem_ctx *c, const void *u, void *w, bool uh, bool wh, double h1, double h2,
                   sem_dtype dt, cudaStream_t s)
{
    const size_t es = (dt == SEM_F64 || dt == SEM_F64_NATIVE) ? sizeof(double) : sizeof(float);
    const int64_t n3 = (int64_t)c->n * c->n * c->n;
    int rc = sem_ensure_stage(c, (size_t)c->nL * es);
    if (rc) return rc;
    AxPipe *P = ax_pipe(c);
    if (!P) return SEM_ERR_NOMEM;
    const int K = c->E >= 2 * SEM_PIPE_CHUNKS ? SEM_PIPE_CHUNKS : 1;
    const int64_t ne = sem_ceil_div(c->E, K);
    char *ud = uh ? (char *)c->stage[0] : (char *)u;
    char *wd = wh ? (char *)c->stage[1] : (char *)w;
    SEM_CUDA(cudaEventRecord(P->start, s));
    SEM_CUDA(cudaStreamWaitEvent(P->in, P->start, 0));
    SEM_CUDA(cudaStreamWaitEvent(P->out, P->start, 0));
    for (int k = 0; k < K; ++k) {
        const int64_t e0 = k * ne, e1 = e0 + ne < c->E ? e0 + ne : c->E;
        if (e0 >= e1) break;
        const size_t off = (size_t)(e0 * n3) * es, bytes = (size_t)((e1 - e0) * n3) * es;
        if (uh) {
            SEM_CUDA(cudaMemcpyAsync(ud + off, (const char *)u + off, bytes, cudaMemcpyHostToDevice, P->in));
            SEM_CUDA(cudaEventRecord(P->ev_in[k], P->in));
            SEM_CUDA(cudaStreamWaitEvent(s, P->ev_in[k], 0));
        }
        sem_ctx sub = *c;  // the chunk's elements and their geometry
        sub.E = e1 - e0;
        sub.nL = (e1 - e0) * n3;
        sub.geo64 = c->geo64 ? c->geo64 + e0 * 7 * n3 : nullptr;
        sub.geo32 = c->geo32 ? c->geo32 + e0 * 7 * n3 : nullptr;
        sub.geodf = c->geodf ? (void *)((char *)c->geodf + e0 * 7 * n3 * 8) : nullptr;
        rc = sem_ax_dev(&sub, ud + off, wd + off, h1, h2, dt, s);
        if (rc) return rc;
        if (wh) {
            SEM_CUDA(cudaEventRecord(P->ev_cmp[k], s));
            SEM_CUDA(cudaStreamWaitEvent(P->out, P->ev_cmp[k], 0));
            SEM_CUDA(cudaMemcpyAsync((char *)w + off, wd + off, bytes, cudaMemcpyDeviceToHost, P->out));
        }
    }
    if (wh) {
        SEM_CUDA(cudaEventRecord(P->done, P->out));
        SEM_CUDA(cudaStreamWaitEvent(s, P->done, 0));
    }
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
}

// The device address of pinned (page-locked, mapped) host memory, else null.
// Under unified addressing every pinned allocation is mapped; on GB300 the
// Grace memory behind it is reached coherently over NVLink-C2C.
static void *mapped_host(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// FP64-accurate operator on pinned host buffers without staging copies: the
// kernel's own loads and stores cross the host link (its u prefetch into L2 is
// off), so transfer and arithmetic overlap at the granularity of the loads.
static int ax_mapped(sem_ctx *c, const void *u, void *w, bool uh, bool wh, double h1, double h2,
                     cudaStream_t s, bool *done)
{
    *done = false;
    const void *du = uh ? mapped_host(u) : u;
    void *dw = wh ? mapped_host(w) : w;
    if (!du || !dw || ((uintptr_t)du | (uintptr_t)dw) % sizeof(double)) return SEM_OK;
    sem_ctx sub = *c;
    sub.u_sysmem = uh ? 1 : 0;
    int rc = sem_ax_dev(&sub, du, dw, h1, h2, SEM_F64, s);
    if (rc) return rc;
    SEM_CUDA(cudaStreamSynchronize(s));
    *done = true;
    return SEM_OK;
}

extern "C" int sem_ax(sem_ctx *c, const void *u, void *w, double h1, double h2, sem_dtype dt,
                      void *stream)
{
    if (!c || !u || !w) return SEM_ERR_ARG;
    if (dt < SEM_F64 || dt > SEM_BF16X3_TC) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool uh = !sem_is_device_ptr(u), wh = !sem_is_device_ptr(w);
    if (uh || wh) {
        if (dt == SEM_F64) {
            bool done = false;
            int rc = ax_mapped(c, u, w, uh, wh, h1, h2, s, &done);
            if (rc || done) return rc;
        }
        return ax_host(c, u, w, uh, wh, h1, h2, dt, s);
    }
    return sem_ax_dev(c, u, w, h1, h2, dt, s);
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
    if (dt < SEM_F64 || dt > SEM_BF16X3_TC || dt == SEM_F64_NATIVE) return SEM_ERR_ARG;
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
    // FP32: three tile shapes; FP64-accurate, even N+1 <= 10: three elements-per-block
    // counts of the folded kernel; otherwise one candidate
    const int nvar = dt == SEM_F32 || (dt == SEM_F64 && c->n % 2 == 0 && c->n <= 12) ||
                             (dt == SEM_F64_NATIVE && c->n % 2 == 0)
                         ? sem_nvariant(dt)
                         : 1;
    if (ms)
        for (int v = 0; v < SEM_NVARIANT; ++v) ms[v] = -1.0;
    if (nvar == 1) {
        *best = 0;
        if (ms) ms[0] = 0.0;
        return sem_set_ax_variant(c->N, dt, 0);
    }
    // the solver workspace of slot 0 (allocated by sem_setup) serves as input
    // and output, its contents being scratch between solves: r and w
    // (FP64-accurate) or r32 and w32 (FP32); u = 0 (the kernels' instruction
    // streams and memory traffic do not depend on the values)
    if (!c->ws[0].r || !c->ws[0].r32) return SEM_ERR_ARG;
    const void *u = dt == SEM_F32 ? (const void *)c->ws[0].r32 : (const void *)c->ws[0].r;
    void *w = dt == SEM_F32 ? (void *)c->ws[0].w32 : (void *)c->ws[0].w;
    cudaStream_t s = 0;
    cudaEvent_t e0, e1;
    SEM_CUDA(cudaEventCreate(&e0));
    SEM_CUDA(cudaEventCreate(&e1));
    SEM_CUDA(cudaMemsetAsync((void *)u, 0, (dt == SEM_F32 ? sizeof(float) : sizeof(double)) * c->nL, s));
    const int saved = sem_ax_variant(c->N, dt);
    auto run = [&](int v) {
        if (dt == SEM_F32)
            return sem_launch_ax_f32_variant(c, v, (const float *)u, (float *)w, 1.0f, 1.0f, s);
        if (dt == SEM_F64_NATIVE)
            return sem_launch_ax_f64_v(c, (const double *)u, (double *)w, 1.0, 1.0, v == 0, s);
        int rc = sem_set_ax_variant(c->N, dt, v);
        return rc ? rc : sem_launch_ax_df(c, (const double *)u, (double *)w, 1.0, 1.0, s);
    };
    double best_ms = 1e300;
    int bi = 0;
    for (int v = 0; v < nvar; ++v) {
        double t = 1e300;
        int rc = run(v);  // warm-up
        if (rc == SEM_OK) {
            SEM_CUDA(cudaEventRecord(e0, s));
            for (int k = 0; k < reps && rc == SEM_OK; ++k) rc = run(v);
            SEM_CUDA(cudaEventRecord(e1, s));
            SEM_CUDA(cudaEventSynchronize(e1));
            float f = 0.f;
            SEM_CUDA(cudaEventElapsedTime(&f, e0, e1));
            t = f / reps;
        }
        if (ms) ms[v] = rc == SEM_OK ? t : -1.0;
        if (rc == SEM_OK && t < best_ms) {
            best_ms = t;
            bi = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms == 1e300) {
        sem_set_ax_variant(c->N, dt, saved);
        return SEM_ERR_CUDA;
    }
    *best = bi;
    return sem_set_ax_variant(c->N, dt, bi);
}
