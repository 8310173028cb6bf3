// noalloc.cu -- a PCG entry point that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code that runs under a memory manager
// that owns the whole device budget (a framework's caching allocator, a plugin
// host, a real-time service that pre-plans every byte) and code that must not
// pay cudaMalloc's implicit device synchronisation.  sem_pcg_solve_noalloc
// serves them: it runs the persistent Jacobi-PCG kernel of sem_pcg_solve in
// its native-FP64 mode (the arithmetic of sem_pcg_solve with inner =
// SEM_F64_NATIVE), without a context, with every scratch vector, partial sum
// and solver state in the file-scope array below.  The caller passes the
// inputs (geometry, right-hand side) and the output (x); nothing is allocated
// by this file.  The call reads the mesh volume back and synchronises the
// caller's stream twice.
#include <math.h>
#include <string.h>

#include <mutex>

#include "solver.cuh"

GsDesc sem_gs_desc(const sem_ctx *c);  // ops.cu

#define SEM_DECL_NP(NPV) int sem_solve_launch_np##NPV(const SolveParams<8> &, int, int, long long, cudaStream_t);
SEM_DECL_NP(2) SEM_DECL_NP(3) SEM_DECL_NP(4) SEM_DECL_NP(5) SEM_DECL_NP(6) SEM_DECL_NP(7)
SEM_DECL_NP(8) SEM_DECL_NP(9) SEM_DECL_NP(10) SEM_DECL_NP(11) SEM_DECL_NP(12) SEM_DECL_NP(13)
SEM_DECL_NP(14) SEM_DECL_NP(15) SEM_DECL_NP(16)
#undef SEM_DECL_NP

typedef int (*noalloc_launch_fn)(const SolveParams<8> &, int, int, long long, cudaStream_t);
static const noalloc_launch_fn k_noalloc_launch[17] = {
    nullptr, nullptr, sem_solve_launch_np2, sem_solve_launch_np3, sem_solve_launch_np4,
    sem_solve_launch_np5, sem_solve_launch_np6, sem_solve_launch_np7, sem_solve_launch_np8,
    sem_solve_launch_np9, sem_solve_launch_np10, sem_solve_launch_np11, sem_solve_launch_np12,
    sem_solve_launch_np13, sem_solve_launch_np14, sem_solve_launch_np15, sem_solve_launch_np16};

// Scratch layout (bytes from the start of the array):
//   [0, HEAD)             solver state: SyncState, PState[8], schedule
//   [HEAD, HEAD + PART)   per-CTA partial sums
//   [.., + TAB)           derivative matrix D (FP64) and the mass sum
//   then 4 FP64 vectors of nL entries: r, p, w, minv
#define NA_HEAD (64 * 1024)
#define NA_GRID_MAX 2048
#define NA_PART ((size_t)NA_GRID_MAX * 8 * 3 * sizeof(double))
#define NA_TAB (4 * 1024)
#define NA_VEC_OFF (NA_HEAD + NA_PART + NA_TAB)
#define NA_BYTES ((size_t)NA_VEC_OFF + (size_t)4 * SEM_NOALLOC_MAX_NODES * sizeof(double))

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NaStateHost {
    SyncState sync;
    PState st[8];
    int sched[8 * 2 + 2];
};
static_assert(sizeof(NaStateHost) <= NA_HEAD, "solver state exceeds its scratch slot");

// Per-device device addresses of the scratch array, looked up once per device
// (with that device current) by the first call there.  A cudaDeviceReset of the
// device reloads the module and leaves the cached address stale, so calls after
// a reset in the same process are not supported.
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[64];

static int noalloc_scratch(unsigned char **out)
{
    int dev = 0;
    SEM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SEM_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        SEM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = (unsigned char *)p;
    }
    *out = g_noalloc_addr[dev];
    return SEM_OK;
}

struct NaTable {
    double D[SEM_NPMAX * SEM_NPMAX];
};

// Writes D into the scratch and sums the mass B (element-blocked geometry,
// component 6) in a fixed order: one block, strided partial sums, then a tree.
__global__ void k_noalloc_prep(NaTable tab, int n, const double *__restrict__ geo, int64_t E,
                               double *__restrict__ Dout, double *__restrict__ vol)
{
    __shared__ double sh[256];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) Dout[t] = tab.D[t];
    const int n3 = n * n * n;
    double s = 0.0;
    for (int64_t e = 0; e < E; ++e)
        for (int l = threadIdx.x; l < n3; l += blockDim.x) s += geo[(e * 7 + 6) * n3 + l];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *vol = sh[0];
}

// Derivative matrix of the GLL basis (host): barycentric form with the
// negative-sum diagonal.  The nodes come from Newton on P_{N+1} - P_{N-1}.
static void noalloc_tables(int N, double *D)
{
    const int n = N + 1;
    double xi[SEM_NPMAX], lam[SEM_NPMAX];
    for (int i = 0; i <= N; ++i) {
        double x = -cos(M_PI * i / N);
        if (i > 0 && i < N) {
            for (int it = 0; it < 60; ++it) {
                double pm = 1.0, pc = x;
                for (int k = 1; k < N; ++k) {
                    double nx = ((2 * k + 1) * x * pc - k * pm) / (k + 1);
                    pm = pc;
                    pc = nx;
                }
                double pn1 = ((2 * N + 1) * x * pc - N * pm) / (N + 1);
                double dx = (pn1 - pm) / ((2 * N + 1) * pc);
                x -= dx;
                if (fabs(dx) < 1e-17) break;
            }
        }
        xi[i] = x;
    }
    for (int i = 0; i < (N + 1) / 2; ++i) {
        double s = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -s;
        xi[N - i] = s;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
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
            D[i * n + j] = (lam[j] / lam[i]) / (xi[i] - xi[j]);
            s += D[i * n + j];
        }
        D[i * n + i] = -s;
    }
}

extern "C" int sem_pcg_solve_noalloc(int N, int nelx, int nely, int nelz, const int periodic[3],
                                     const double *geom, const double *b, double *x, double h1,
                                     double h2, const sem_solve_opts *opts, sem_solve_info *info,
                                     void *stream)
{
    if (N < 1 || N > SEM_NMAX || nelx < 1 || nely < 1 || nelz < 1 || !periodic || !geom || !b ||
        !x || !info)
        return SEM_ERR_ARG;
    sem_solve_opts o;
    sem_solve_opts_default(&o);
    if (opts) o = *opts;
    if ((o.inner != SEM_F64 && o.inner != SEM_F64_NATIVE) || !(o.tol >= 0) || o.maxit < 0)
        return SEM_ERR_ARG;
    if (!(h1 >= 0) || !(h2 >= 0) || (h1 == 0 && h2 == 0)) return SEM_ERR_ARG;
    const int n = N + 1;
    const int64_t E = (int64_t)nelx * nely * nelz;
    const int64_t nL = E * n * n * n;
    if (nL > SEM_NOALLOC_MAX_NODES) return SEM_ERR_TOO_LARGE;
    if (!sem_is_device_ptr(geom) || !sem_is_device_ptr(b) || !sem_is_device_ptr(x)) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    int dev = 0, sms = 0;
    SEM_CUDA(cudaGetDevice(&dev));
    SEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if ((long long)sms * SEM_SOLVE_MAX_GRID_PER_SM > NA_GRID_MAX) return SEM_ERR_ARG;

    NaStateHost *state = (NaStateHost *)base;
    double *partials = (double *)(base + NA_HEAD);
    double *Dd = (double *)(base + NA_HEAD + NA_PART);
    double *vol = Dd + SEM_NPMAX * SEM_NPMAX;
    double *vec = (double *)(base + NA_VEC_OFF);

    NaTable tab;
    memset(&tab, 0, sizeof(tab));
    noalloc_tables(N, tab.D);
    k_noalloc_prep<<<1, 256, 0, s>>>(tab, n, geom, E, Dd, vol);
    SEM_CHECK_LAUNCH();
    double volume = 0.0;
    SEM_CUDA(cudaMemcpyAsync(&volume, vol, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));

    sem_ctx shape;  // only the fields sem_gs_desc reads
    memset(&shape, 0, sizeof(shape));
    shape.N = N;
    shape.n = n;
    shape.nelx = nelx; shape.nely = nely; shape.nelz = nelz;
    for (int d = 0; d < 3; ++d) shape.periodic[d] = periodic[d] ? 1 : 0;
    shape.ngx = nelx * N + (shape.periodic[0] ? 0 : 1);
    shape.ngy = nely * N + (shape.periodic[1] ? 0 : 1);
    shape.ngz = nelz * N + (shape.periodic[2] ? 0 : 1);
    shape.nG = (int64_t)shape.ngx * shape.ngy * shape.ngz;

    SolveParams<8> prm;
    memset(&prm, 0, sizeof(prm));
    prm.nprob = 1;
    prm.abs_tol = o.abs_tol;
    prm.maxit = o.maxit;
    prm.max_outer = o.max_outer;
    prm.tol = o.tol;
    prm.inner_tol = o.inner_tol;
    prm.timeout_ns = (long long)((o.wait_timeout_s > 0 ? o.wait_timeout_s : 10.0) * 1e9);
    prm.sync = &state->sync;
    prm.st = state->st;
    prm.sched = state->sched;
    prm.partials = partials;
    ProbDesc &d = prm.prob[0];
    d.n = n;
    d.NE = (256 / (n * n)) > 0 ? 256 / (n * n) : 1;
    d.NE32 = d.NE;
    d.singular = (h2 == 0.0);
    d.E = E;
    d.nL = nL;
    d.nG = shape.nG;
    d.gs = sem_gs_desc(&shape);
    d.volume = volume;
    d.h1 = h1;
    d.h2 = h2;
    d.geo64 = geom;
    d.D64 = Dd;
    d.b = b;
    d.x = x;
    d.r = vec;
    d.p = vec + nL;
    d.w = vec + 2 * nL;
    d.minv = vec + 3 * nL;

    // the array keeps the previous call's contents: the solver state must start at zero
    SEM_CUDA(cudaMemsetAsync(state, 0, sizeof(NaStateHost), s));
    rc = k_noalloc_launch[n](prm, MODE_F64N, sms, (nL + SEM_SOLVE_THREADS - 1) / SEM_SOLVE_THREADS, s);
    if (rc) return rc;
    NaStateHost h;
    SEM_CUDA(cudaMemcpyAsync(&h, state, sizeof(NaStateHost), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    info->status = h.sync.err ? h.sync.err : h.st[0].status;
    info->iters = h.st[0].iters;
    info->outer_iters = 0;
    info->final_rnorm = h.st[0].rnorm;
    info->bnorm = h.st[0].bnorm;
    return info->status;
}
