// tgv.cu -- Taylor-Green vortex stepper: BDF3/EXT3 P_N-P_N with 3/2 dealiasing.
//
// One step (Sec. 3: "P_N-P_N", "fixed third-order time integration",
// "dealiasing enabled"; hotspots of Sec. 1.1 Fig. 3), order q = min(step+1, 3):
//   1. C^n_c   = weak dealiased (u^n . grad) u^n_c on M^3 Gauss points,
//                M = ceil(3(N+1)/2)                              (k_convect)
//   2. F_c     = -sum_j a_j C^{n+1-j}_c                          (k_tgv_F)
//   3. g_c     = dssum(F_c) / dssum(B) + sum_j b_j u^{n+1-j}_c / dt
//                                                                (k_tgv_g, unique nodes)
//   4. A p     = dssum( sum_a D_a^T ( B sum_c (dr_a/dx_c) g_c ) )  (k_tgv_divg + PCG)
//   5. (nu A + b0/dt B) u_c = dssum( F_c + B (sum_j b_j u_c/dt - dp/dx_c) )
//                                                   (k_tgv_vrhs + 3-problem batched PCG)
//   6. shift histories; KE and enstrophy into a device log      (k_tgv_diag_*)
// Precision policy (Sec. 2, Fig. 2): the rule in force at a step selects the
// convection precision (FP64, FP32, or FP16/BF16 operands with FP32
// accumulation), the inner precision of the velocity and pressure solves, and
// whether the stored state (velocity and convection histories, pressure) is
// rounded to FP32 values where it is stored.
// Histories, right-hand sides and diagnostics are FP64.  With op = SEM_F32 the
// convective term is computed in FP32; the solves use the precision of the
// options passed (the default pressure options then select an FP32 inner PCG
// inside FP64 refinement; the velocity Helmholtz solves, a few iterations per
// step, stay FP64 unless their options ask otherwise).  Steady-state steps (q = 3) are captured once into
// a CUDA graph and replayed.  Orders N <= 9.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "df64.cuh"
#include "gs.cuh"

GsDesc sem_gs_desc(const sem_ctx *c);
int sem_run_geometry(sem_ctx *c, double *xyz, bool with_jinv, cudaStream_t s);
int sem_alloc_ws(sem_ctx *c, int slot);
int sem_dssum_dev(sem_ctx *c, void *u, sem_dtype dt, cudaStream_t s);
int sem_ax_dev(sem_ctx *c, const void *u, void *w, double h1, double h2, sem_dtype dt, cudaStream_t s);
int sem_pcg_solve_dev(sem_ctx *c, int slot, const double *b, double *x, double h1, double h2,
                      const sem_solve_opts &o, cudaStream_t s);
int sem_pcg_solve_dev_batch(sem_ctx *c, int np, const double *const *b, double *const *x, double h1,
                            double h2, const sem_solve_opts &o, cudaStream_t s, int slot0);
const void *sem_solve_state_ptr(const sem_ctx *c, int p, int *iters_off, int *status_off);
int sem_gmres_solve_dev(sem_hsmg *H, int precond, const double *b_in, double *x, const sem_solve_opts &o,
                        int m, sem_solve_info *info, cudaStream_t s, int x_zero);
const void *sem_solve_sync_ptr(const sem_ctx *c);

#define TGV_LOG 4096

struct TgvLogEntry {
    double t, ke, en;
    int iters[4];
    int status;
    int pad;
    double dt, cfl;   // the step's size and the CFL number of its new velocity
};

struct TgvDev {       // device-side counters
    long long count;  // entries written so far
    double t;
    double cfl;       // CFL number of the latest step
};

struct sem_tgv {
    sem_ctx *c;
    double nu, dt;
    sem_dtype op;          // convection precision in force
    sem_dtype storage;     // stored-state precision in force (SEM_F64 or SEM_F32)
    sem_solve_opts vo, po; // solve options in force
    sem_dtype op0, vin0, pin0;  // the precisions given to sem_tgv_init
    sem_tgv_policy rules[SEM_TGV_MAX_RULES];
    int nrules, cur_rule;  // cur_rule: -1 = init precisions, -2 = not applied yet
    // projection of the pressure solve (0 vectors = off)
    int proj_max;
    double *pX, *pBX;      // [proj_max][nL]: A-orthonormal basis and A times it (assembled)
    double *pw, *pxb, *pbq, *pdx, *padx;  // 1/multiplicity, projection, remainder RHS, solve, A v
    double *pcoef;         // device scalars: coefficients [TGV_PMAX], norms [2]
    double *ppart;         // per-block partial dots [TGV_PBLK][TGV_PMAX]
    int *pint;             // device ints: basis size L, 1, restart flag
    int step, M;
    double t;
    double hist_dt[2];        // sizes of the last two steps (most recent first)
    double cfl_target, dt_max; // adaptive step when cfl_target > 0
    TgvDev *hdev;             // pinned host copy of the counters
    // pressure solver: 0 Jacobi-PCG (persistent kernel), 1 flexible GMRES + HSMG
    int psolver, prestart;
    sem_hsmg *hsmg;
    sem_solve_info pinfo;     // the last GMRES pressure solve
    double *u[3][3], *C[3][3], *p, *unew[3], *F[3], *g[3], *bp, *rhs[3];
    // FP32 storage (rp = fp32): the velocity and convection histories live in
    // these FP32 buffers instead of u and C while storage == SEM_F32
    float *u32[3][3], *C32[3][3];
    float *block32;    // one allocation for them (made by the first rule that needs it)
    double *part;      // [E][2]
    double *tab64;     // eta[M], wq[M], J[M*n]
    float *tab32;
    df64 *tabdf;       // the same tables as float pairs (FP64-accurate convection)
    df64 *jinvdf;      // J^{-1} as float pairs, [E][9][n^3]
    TgvLogEntry *log;  // device ring
    TgvLogEntry *hlog; // pinned host copy
    TgvDev *dev;
    cudaGraphExec_t graph;
    cudaStream_t graph_stream;
    int graph_state;   // 0 not tried, 1 ready, -1 unavailable
    int graph_warm;    // a steady step ran directly since the last (re)capture was needed
    double *block;     // one allocation for all fields
};

// ---------------------------------------------------------------------------
// 1-D tables of the dealiasing grid (host)
// ---------------------------------------------------------------------------

// Gauss-Legendre points and weights by Newton on P_M.
static void gl_table(int M, double *eta, double *wq)
{
    for (int q = 0; q < M; ++q) {
        double x = -cos(M_PI * (q + 0.75) / (M + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < M; ++k) {
                double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
                p0 = p1;
                p1 = p2;
            }
            dp = M * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 1; k < M; ++k) {
            double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
            p0 = p1;
            p1 = p2;
        }
        dp = M * (x * p1 - p0) / (x * x - 1.0);
        eta[q] = x;
        wq[q] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    for (int q = 0; q < M / 2; ++q) {
        double s = 0.5 * (eta[M - 1 - q] - eta[q]);
        eta[q] = -s;
        eta[M - 1 - q] = s;
        double w = 0.5 * (wq[q] + wq[M - 1 - q]);
        wq[q] = wq[M - 1 - q] = w;
    }
    if (M % 2 == 1) eta[M / 2] = 0.0;
}

// J[q][j] = l_j(eta_q) on the GLL nodes xi (barycentric form).
static void interp_table(int n, const double *xi, int M, const double *eta, double *J)
{
    double lam[SEM_NPMAX];
    for (int j = 0; j < n; ++j) {
        double pr = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) pr *= (xi[j] - xi[k]);
        lam[j] = 1.0 / pr;
    }
    for (int q = 0; q < M; ++q) {
        int hit = -1;
        for (int j = 0; j < n; ++j)
            if (eta[q] == xi[j]) hit = j;
        double den = 0.0;
        for (int j = 0; j < n; ++j)
            if (hit < 0) den += lam[j] / (eta[q] - xi[j]);
        for (int j = 0; j < n; ++j)
            J[q * n + j] = hit >= 0 ? (j == hit ? 1.0 : 0.0) : (lam[j] / (eta[q] - xi[j])) / den;
    }
}

// ---------------------------------------------------------------------------
// Dealiased convective term
// ---------------------------------------------------------------------------

// Stored fields (velocity and convection histories) are FP64, or FP32 under
// FP32 storage; s32 selects the type at run time (warp-uniform), values are
// widened to FP64 on load and rounded to nearest on store.
__device__ __forceinline__ double ld_fs(const void *p, int64_t q, int s32)
{
    return s32 ? (double)((const float *)p)[q] : ((const double *)p)[q];
}

__device__ __forceinline__ void st_fs(void *p, int64_t q, double v, int s32)
{
    if (s32) ((float *)p)[q] = __double2float_rn(v);
    else ((double *)p)[q] = v;
}

template <int NP>
struct ConvCfg {
    static constexpr int M = (3 * NP + 1) / 2;
    static constexpr int N3 = NP * NP * NP, M3 = M * M * M;
    static constexpr int T1 = NP * NP * M, T2 = NP * M * M;
    template <typename T>
    static constexpr size_t smem()
    {
        return sizeof(T) * (size_t)(3 * N3 + 3 * N3 + 3 * M3 + M3 + T1 + T2 + 2 * (M * NP + NP * NP) + M + M + 32);
    }
};

struct ConvArgs {
    const void *u[3];  // stored fields (FP32 when s32)
    void *C[3];
    int s32;
    const void *jinv;  // [E][9][n3], FP64 or FP32 per T
    const double *vert;
    const void *D;     // n*n (T)
    const void *tab;   // eta[M], wq[M], J[M*n] (T)
    int nelx, nely;
    int64_t E;
};

// Operand rounding of the 16-bit convection overrides: R16 = 1 FP16, 2 BF16.
template <int R16, typename T>
__device__ __forceinline__ T rnd16(T x)
{
    if constexpr (R16 == 1)
        return (T)__half2float(__float2half_rn((float)x));
    else if constexpr (R16 == 2)
        return (T)__bfloat162float(__float2bfloat16_rn((float)x));
    else
        return x;
}

// v = (J x J x J) in  (n^3 -> M^3); fin(q, value) receives each output.  sJT is
// J transposed ([l][q]): the first stage's 32 lanes then read consecutive words
// (J row-major would put 12 rows 8 words apart on the same banks).
template <int NP, typename T, int R16, class Fin>
__device__ __forceinline__ void interp_fwd(const T *in, T *st1, T *st2, const T *sJ, const T *sJT, Fin fin)
{
    using C = ConvCfg<NP>;
    constexpr int M = C::M;
    for (int t = threadIdx.x; t < C::T1; t += blockDim.x) {
        const int q1 = t % M, j = (t / M) % NP, k = t / (M * NP);
        T s = 0;
#pragma unroll
        for (int l = 0; l < NP; ++l) s = fma(sJT[l * M + q1], in[(k * NP + j) * NP + l], s);
        st1[t] = rnd16<R16>(s);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C::T2; t += blockDim.x) {
        const int q1 = t % M, q2 = (t / M) % M, k = t / (M * M);
        T s = 0;
#pragma unroll
        for (int l = 0; l < NP; ++l) s = fma(sJ[q2 * NP + l], st1[(k * NP + l) * M + q1], s);
        st2[t] = rnd16<R16>(s);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C::M3; t += blockDim.x) {
        const int q1 = t % M, q2 = (t / M) % M, q3 = t / (M * M);
        T s = 0;
#pragma unroll
        for (int l = 0; l < NP; ++l) s = fma(sJ[q3 * NP + l], st2[(l * M + q2) * M + q1], s);
        fin(t, s);
    }
    __syncthreads();
}

// out = (J^T x J^T x J^T) f  (M^3 -> n^3).
template <int NP, typename T, int R16, class Fin>
__device__ __forceinline__ void interp_bwd(const T *f, T *st1, T *st2, const T *sJ, Fin fin)
{
    using C = ConvCfg<NP>;
    constexpr int M = C::M;
    for (int t = threadIdx.x; t < C::T2; t += blockDim.x) {  // [q3][q2][i]
        const int i = t % NP, q2 = (t / NP) % M, q3 = t / (NP * M);
        T s = 0;
#pragma unroll 4
        for (int q = 0; q < M; ++q) s = fma(sJ[q * NP + i], f[(q3 * M + q2) * M + q], s);
        st2[t] = rnd16<R16>(s);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C::T1; t += blockDim.x) {  // [q3][j][i]
        const int i = t % NP, j = (t / NP) % NP, q3 = t / (NP * NP);
        T s = 0;
#pragma unroll 4
        for (int q = 0; q < M; ++q) s = fma(sJ[q * NP + j], st2[(q3 * M + q) * NP + i], s);
        st1[t] = rnd16<R16>(s);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C::N3; t += blockDim.x) {
        const int i = t % NP, j = (t / NP) % NP, k = t / (NP * NP);
        T s = 0;
#pragma unroll 4
        for (int q = 0; q < M; ++q) s = fma(sJ[q * NP + k], st1[(q * NP + j) * NP + i], s);
        fin(t, s);
    }
    __syncthreads();
}

template <int NP, typename T, int R16>
__global__ void __launch_bounds__(256) k_convect(ConvArgs a)
{
    using C = ConvCfg<NP>;
    constexpr int M = C::M, N3 = C::N3, M3 = C::M3;
    extern __shared__ __align__(16) unsigned char smem[];
    T *su = reinterpret_cast<T *>(smem);  // [3][N3]
    T *sg = su + 3 * N3;                  // [3][N3]
    T *sfu = sg + 3 * N3;                 // [3][M3] : W|J| u_d on the fine grid
    T *sf = sfu + 3 * M3;                 // [M3]
    T *st1 = sf + M3, *st2 = st1 + C::T1;
    T *sJ = st2 + C::T2, *sD = sJ + M * NP, *seta = sD + NP * NP, *sw = seta + M;
    T *sc = sw + M;                       // trilinear coefficients [8][3]
    T *sJT = sc + 32, *sDT = sJT + M * NP;  // J and D transposed (conflict-free lane patterns)
    const T *D = (const T *)a.D, *tab = (const T *)a.tab;
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sD[t] = rnd16<R16>(D[t]);
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        seta[t] = tab[t];
        sw[t] = tab[M + t];
    }
    for (int t = threadIdx.x; t < M * NP; t += blockDim.x) {
        const T v = rnd16<R16>(tab[2 * M + t]);
        sJ[t] = v;
        sJT[(t % NP) * M + t / NP] = v;
    }
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sDT[(t % NP) * NP + t / NP] = rnd16<R16>(D[t]);
    const T *jinv = (const T *)a.jinv;
    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        __syncthreads();
        const int64_t off = e * N3;
        for (int t = threadIdx.x; t < 3 * N3; t += blockDim.x)
            su[t] = rnd16<R16>((T)ld_fs(a.u[t / N3], off + t % N3, a.s32));
        if (threadIdx.x < 24) {  // x = c0 + c1 r + c2 s + c3 t + c4 rs + c5 rt + c6 st + c7 rst
            const int m = threadIdx.x / 3, d = threadIdx.x % 3;
            const int ex = (int)(e % a.nelx), ey = (int)((e / a.nelx) % a.nely),
                      ez = (int)(e / ((int64_t)a.nelx * a.nely));
            double s = 0.0;
            for (int cz = 0; cz < 2; ++cz)
                for (int cy = 0; cy < 2; ++cy)
                    for (int cx = 0; cx < 2; ++cx) {
                        const int64_t vi = ((int64_t)(ez + cz) * (a.nely + 1) + (ey + cy)) * (a.nelx + 1) + (ex + cx);
                        const double sx = cx ? 1.0 : -1.0, sy = cy ? 1.0 : -1.0, sz = cz ? 1.0 : -1.0;
                        const double sg8[8] = {1.0, sx, sy, sz, sx * sy, sx * sz, sy * sz, sx * sy * sz};
                        s += sg8[m] * 0.125 * a.vert[vi * 3 + d];
                    }
            sc[m * 3 + d] = (T)s;
        }
        __syncthreads();
        // fine-grid velocity, scaled by the quadrature weight and |J|
        for (int d = 0; d < 3; ++d)
            interp_fwd<NP, T, R16>(su + d * N3, st1, st2, sJ, sJT, [&](int q, T v) { sfu[d * M3 + q] = v; });
        for (int q = threadIdx.x; q < M3; q += blockDim.x) {
            const int q1 = q % M, q2 = (q / M) % M, q3 = q / (M * M);
            const T r = seta[q1], s = seta[q2], t = seta[q3];
            T J[3][3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                J[d][0] = sc[1 * 3 + d] + sc[4 * 3 + d] * s + sc[5 * 3 + d] * t + sc[7 * 3 + d] * s * t;
                J[d][1] = sc[2 * 3 + d] + sc[4 * 3 + d] * r + sc[6 * 3 + d] * t + sc[7 * 3 + d] * r * t;
                J[d][2] = sc[3 * 3 + d] + sc[5 * 3 + d] * r + sc[6 * 3 + d] * s + sc[7 * 3 + d] * r * s;
            }
            const T det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                          J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            const T wd = sw[q1] * sw[q2] * sw[q3] * det;
            sfu[q] = rnd16<R16>(sfu[q] * wd);
            sfu[M3 + q] = rnd16<R16>(sfu[M3 + q] * wd);
            sfu[2 * M3 + q] = rnd16<R16>(sfu[2 * M3 + q] * wd);
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c) {
            // physical gradient of u_c on the GLL nodes
            const T *uc = su + c * N3;
            for (int pn = threadIdx.x; pn < N3; pn += blockDim.x) {
                const int i = pn % NP, j = (pn / NP) % NP, k = pn / (NP * NP);
                T gr = 0, gs = 0, gt = 0;
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    gr = fma(sDT[l * NP + i], uc[(k * NP + j) * NP + l], gr);
                    gs = fma(sD[j * NP + l], uc[(k * NP + l) * NP + i], gs);
                    gt = fma(sD[k * NP + l], uc[(l * NP + j) * NP + i], gt);
                }
                const T *ji = jinv + e * 9 * N3 + pn;
                gr = rnd16<R16>(gr);
                gs = rnd16<R16>(gs);
                gt = rnd16<R16>(gt);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    sg[d * N3 + pn] = rnd16<R16>(rnd16<R16>(ji[(0 * 3 + d) * N3]) * gr +
                                                 rnd16<R16>(ji[(1 * 3 + d) * N3]) * gs +
                                                 rnd16<R16>(ji[(2 * 3 + d) * N3]) * gt);
            }
            for (int q = threadIdx.x; q < M3; q += blockDim.x) sf[q] = 0;
            __syncthreads();
            for (int d = 0; d < 3; ++d)
                interp_fwd<NP, T, R16>(sg + d * N3, st1, st2, sJ, sJT,
                                  [&](int q, T v) { sf[q] = fma(sfu[d * M3 + q], rnd16<R16>(v), sf[q]); });
            if (R16) {
                __syncthreads();
                for (int q = threadIdx.x; q < M3; q += blockDim.x) sf[q] = rnd16<R16>(sf[q]);
                __syncthreads();
            }
            void *Cc = a.C[c];
            interp_bwd<NP, T, R16>(sf, st1, st2, sJ, [&](int pn, T v) { st_fs(Cc, off + pn, (double)v, a.s32); });
        }
    }
}

// ---------------------------------------------------------------------------
// Pointwise / element kernels of the step
// ---------------------------------------------------------------------------

struct Coef {
    double a[3], b[3], b0, dt;
};

struct FArgs {
    const void *C[3][3];  // [level][comp], stored fields
    double *F[3];
    int s32;
};

// Initial guess of the velocity solves: u_c^* = sum_j a_j u_c^{n+1-j} (the EXT
// weights of the step), from the stored histories into the FP64 iterate.
struct XArgs {
    const void *u[3][3];  // [level][comp], stored fields
    double *x[3];
    int s32;
};

__global__ void k_tgv_ext(XArgs a, Coef k, int64_t nL)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nL) return;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        a.x[c][q] = k.a[0] * ld_fs(a.u[0][c], q, a.s32) + k.a[1] * ld_fs(a.u[1][c], q, a.s32) +
                    k.a[2] * ld_fs(a.u[2][c], q, a.s32);
}

__global__ void k_tgv_F(FArgs a, Coef k, int64_t nL)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nL) return;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        a.F[c][q] = -(k.a[0] * ld_fs(a.C[0][c], q, a.s32) + k.a[1] * ld_fs(a.C[1][c], q, a.s32) +
                      k.a[2] * ld_fs(a.C[2][c], q, a.s32));
}

struct GArgs {
    const double *F[3];
    const void *u[3][3];  // [level][comp], stored fields
    double *g[3];
    const double *geo64;
    GsDesc gs;
    Coef k;
    int s32;
};

// g_c = dssum(F_c) / dssum(B) + sum_j b_j u^{n+1-j}_c / dt at every copy.
__global__ void k_tgv_g(GArgs a)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= a.gs.nG) return;
    int64_t idx[8];
    const int m = gs_copies(a.gs, g, idx);
    const int n3 = a.gs.n * a.gs.n * a.gs.n;
    double bs = 0.0;
    for (int t = 0; t < m; ++t) {
        const int64_t e = idx[t] / n3;
        bs += a.geo64[(e * 7 + 6) * n3 + (idx[t] - e * n3)];
    }
    const int64_t f = idx[0];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int t = 0; t < m; ++t) s += a.F[c][idx[t]];
        const double hist = a.k.b[0] * ld_fs(a.u[0][c], f, a.s32) + a.k.b[1] * ld_fs(a.u[1][c], f, a.s32) +
                            a.k.b[2] * ld_fs(a.u[2][c], f, a.s32);
        const double v = s / bs + hist / a.k.dt;
        for (int t = 0; t < m; ++t) a.g[c][idx[t]] = v;
    }
}

// bp = sum_a D_a^T ( B sum_c (dr_a/dx_c) g_c )   (local, one block per element)
// T = double, or df64 (FP64-accurate on the FP32 pipes): jinv, geo and D are
// then the float-pair copies; g and bp stay FP64.
template <int NP, typename T>
__global__ void k_tgv_divg(const double *g0, const double *g1, const double *g2,
                           const T *jinv, const T *geo, const T *D, double *bp, int64_t E)
{
    constexpr int N3 = NP * NP * NP;
    __shared__ T sh[3 * N3];
    __shared__ T sD[NP * NP];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sD[t] = D[t];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        const int64_t off = e * N3;
        for (int pn = threadIdx.x; pn < N3; pn += blockDim.x) {
            const T gv[3] = {T(g0[off + pn]), T(g1[off + pn]), T(g2[off + pn])};
            const T bm = geo[(e * 7 + 6) * N3 + pn];
            const T *ji = jinv + e * 9 * N3 + pn;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                sh[a * N3 + pn] = bm * (ji[(a * 3 + 0) * N3] * gv[0] + ji[(a * 3 + 1) * N3] * gv[1] +
                                        ji[(a * 3 + 2) * N3] * gv[2]);
        }
        __syncthreads();
        for (int pn = threadIdx.x; pn < N3; pn += blockDim.x) {
            const int i = pn % NP, j = (pn / NP) % NP, k = pn / (NP * NP);
            T s = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                s = fma(sD[l * NP + i], sh[0 * N3 + (k * NP + j) * NP + l], s);
                s = fma(sD[l * NP + j], sh[1 * N3 + (k * NP + l) * NP + i], s);
                s = fma(sD[l * NP + k], sh[2 * N3 + (l * NP + j) * NP + i], s);
            }
            bp[off + pn] = (double)s;
        }
    }
}

struct VArgs {
    const double *F[3];
    const void *u[3][3];  // stored fields
    int s32;
    const double *p;
    const double *jinv, *geo64, *D;
    double *rhs[3];
    Coef k;
    int64_t E;
};

// rhs_c = F_c + B ( sum_j b_j u_c / dt - dp/dx_c )   (local, one block per element)
template <int NP>
__global__ void k_tgv_vrhs(VArgs a)
{
    constexpr int N3 = NP * NP * NP;
    __shared__ double sp[N3];
    __shared__ double sD[NP * NP];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sD[t] = a.D[t];
    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        __syncthreads();
        const int64_t off = e * N3;
        for (int pn = threadIdx.x; pn < N3; pn += blockDim.x) sp[pn] = a.p[off + pn];
        __syncthreads();
        for (int pn = threadIdx.x; pn < N3; pn += blockDim.x) {
            const int i = pn % NP, j = (pn / NP) % NP, k = pn / (NP * NP);
            double gr = 0, gs = 0, gt = 0;
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                gr += sD[i * NP + l] * sp[(k * NP + j) * NP + l];
                gs += sD[j * NP + l] * sp[(k * NP + l) * NP + i];
                gt += sD[k * NP + l] * sp[(l * NP + j) * NP + i];
            }
            const double *ji = a.jinv + e * 9 * N3 + pn;
            const double bm = a.geo64[(e * 7 + 6) * N3 + pn];
            const int64_t q = off + pn;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double dpdx = ji[(0 * 3 + c) * N3] * gr + ji[(1 * 3 + c) * N3] * gs +
                                    ji[(2 * 3 + c) * N3] * gt;
                const double hist = a.k.b[0] * ld_fs(a.u[0][c], q, a.s32) + a.k.b[1] * ld_fs(a.u[1][c], q, a.s32) +
                                    a.k.b[2] * ld_fs(a.u[2][c], q, a.s32);
                a.rhs[c][q] = a.F[c][q] + bm * (hist / a.k.dt - dpdx);
            }
        }
    }
}

// Per-element sum of B|u|^2 and B|curl u|^2.
// T as in k_tgv_divg: the gradients, the vorticity and both integrals per
// element in T; the block sums in FP64.
// With them, the element's largest sum_a |U_a| / dxi_a over its nodes (U_a =
// sum_c (dr_a/dx_c) u_c, dxi_a the GLL gap at the node's index along a; the
// CFL number per unit step, Sec. 3), in FP64 from the T-accurate U_a.
struct GapInv {
    double v[SEM_NPMAX];
};

template <int NP, typename T>
__global__ void k_tgv_diag_part(const void *u0, const void *u1, const void *u2, int s32,
                                const T *jinv, const T *geo, const T *D, GapInv ig, double *part, int64_t E)
{
    constexpr int N3 = NP * NP * NP;
    __shared__ T su[3 * N3];
    __shared__ T sD[NP * NP];
    __shared__ double sred[3 * 32];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sD[t] = D[t];
    const void *uu[3] = {u0, u1, u2};
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        __syncthreads();
        const int64_t off = e * N3;
        for (int t = threadIdx.x; t < 3 * N3; t += blockDim.x) su[t] = T(ld_fs(uu[t / N3], off + t % N3, s32));
        __syncthreads();
        T tke = 0, ten = 0;
        double cmax = 0.0;
        for (int pn = threadIdx.x; pn < N3; pn += blockDim.x) {
            const int i = pn % NP, j = (pn / NP) % NP, k = pn / (NP * NP);
            const T *ji = jinv + e * 9 * N3 + pn;
            {
                const int ia[3] = {i, j, k};
                double cn = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const T U = fma(ji[(a * 3 + 0) * N3], su[pn],
                                    fma(ji[(a * 3 + 1) * N3], su[N3 + pn], ji[(a * 3 + 2) * N3] * su[2 * N3 + pn]));
                    cn += fabs((double)U) * ig.v[ia[a]];
                }
                cmax = fmax(cmax, cn);
            }
            T du[3][3];  // du[c][d] = du_c / dx_d
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T *uc = su + c * N3;
                T gr = 0, gs = 0, gt = 0;
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    gr = fma(sD[i * NP + l], uc[(k * NP + j) * NP + l], gr);
                    gs = fma(sD[j * NP + l], uc[(k * NP + l) * NP + i], gs);
                    gt = fma(sD[k * NP + l], uc[(l * NP + j) * NP + i], gt);
                }
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    du[c][d] = fma(ji[(0 * 3 + d) * N3], gr, fma(ji[(1 * 3 + d) * N3], gs, ji[(2 * 3 + d) * N3] * gt));
            }
            const T wx = du[2][1] - du[1][2], wy = du[0][2] - du[2][0], wz = du[1][0] - du[0][1];
            const T bm = geo[(e * 7 + 6) * N3 + pn];
            tke = fma(bm, fma(su[pn], su[pn], fma(su[N3 + pn], su[N3 + pn], su[2 * N3 + pn] * su[2 * N3 + pn])), tke);
            ten = fma(bm, fma(wx, wx, fma(wy, wy, wz * wz)), ten);
        }
        double ke = (double)tke, en = (double)ten;
        for (int o = 16; o > 0; o >>= 1) {
            ke += __shfl_xor_sync(0xffffffffu, ke, o);
            en += __shfl_xor_sync(0xffffffffu, en, o);
            cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            sred[3 * (threadIdx.x >> 5)] = ke;
            sred[3 * (threadIdx.x >> 5) + 1] = en;
            sred[3 * (threadIdx.x >> 5) + 2] = cmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0, m = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a += sred[3 * w];
                b += sred[3 * w + 1];
                m = fmax(m, sred[3 * w + 2]);
            }
            part[3 * e] = a;
            part[3 * e + 1] = b;
            part[3 * e + 2] = m;
        }
    }
}

// Fixed-order sum of the element partials into the log (and the largest CFL
// rate times dt); advances time and count.
__global__ void k_tgv_diag_final(const double *part, int64_t E, double V, double dt, TgvDev *dv,
                                 TgvLogEntry *log, int advance)
{
    __shared__ double s[3][256];
    double a = 0.0, b = 0.0, m = 0.0;
    for (int64_t e = threadIdx.x; e < E; e += blockDim.x) {
        a += part[3 * e];
        b += part[3 * e + 1];
        m = fmax(m, part[3 * e + 2]);
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        TgvLogEntry &L = log[dv->count % TGV_LOG];
        if (advance) dv->t += dt;
        L.t = dv->t;
        L.ke = s[0][0] / (2.0 * V);
        L.en = s[1][0] / (2.0 * V);
        L.dt = dt;
        L.cfl = dt * s[2][0];
        if (advance) {
            dv->cfl = L.cfl;
            dv->count += 1;
        }
    }
}

// Copies solver iteration counts / status of problems p0..p0+np-1 into the current log entry.
__global__ void k_tgv_log_iters(const char *state, int stride, int iters_off, int status_off,
                                const int *sync_err, int slot0, int np, TgvDev *dv,
                                TgvLogEntry *log, int reset)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    TgvLogEntry &L = log[dv->count % TGV_LOG];
    if (reset) L.status = 0;
    for (int p = 0; p < np; ++p) {
        const char *S = state + (size_t)p * stride;
        L.iters[slot0 + p] = *(const int *)(S + iters_off);
        int st = *sync_err ? *sync_err : *(const int *)(S + status_off);
        if (st != 0 && L.status == 0) L.status = st;
    }
}

// Copy n values between FP64 and FP32 buffers (narrowing rounds to nearest).
__global__ void k_conv_f64_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = __double2float_rn(a[t]);
}

__global__ void k_conv_f32_f64(const float *__restrict__ a, double *__restrict__ b, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (double)a[t];
}

// Iterations and status of a solve known on the host (GMRES) into log slot `slot`.
__global__ void k_tgv_log_host(TgvDev *dv, TgvLogEntry *log, int slot, int iters, int status, int reset)
{
    TgvLogEntry &L = log[dv->count % TGV_LOG];
    if (reset) L.status = 0;
    L.iters[slot] = iters;
    if (status != 0 && L.status == 0) L.status = status;
}

// FP64 values as float pairs (hi = round(v), lo = round(v - hi)).
__global__ void k_split_df64(const double *__restrict__ a, df64 *__restrict__ out, int64_t n)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) out[t] = df64(a[t]);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <int NP>
static size_t conv_smem(bool f32)
{
    return f32 ? ConvCfg<NP>::template smem<float>() : ConvCfg<NP>::template smem<double>();
}

template <int NP, typename T, int R16>
static int run_convect(const ConvArgs &a, int grid, size_t smem, cudaStream_t s)
{
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(k_convect<NP, T, R16>, smem, attr));
    k_convect<NP, T, R16><<<grid, 256, smem, s>>>(a);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

// The stored fields in force: FP32 buffers under FP32 storage, else FP64.
static bool stored32(const sem_tgv *T) { return T->storage == SEM_F32; }
static void *fu(const sem_tgv *T, int l, int c) { return stored32(T) ? (void *)T->u32[l][c] : (void *)T->u[l][c]; }
static void *fC(const sem_tgv *T, int l, int c) { return stored32(T) ? (void *)T->C32[l][c] : (void *)T->C[l][c]; }

static unsigned conv_grid(int64_t n)
{
    const int64_t b = sem_ceil_div(n, 256);
    return (unsigned)(b < 65535 * 8 ? b : 65535 * 8);
}

// Convective term of history level `level` (stored velocity -> stored C).
template <int NP>
static int launch_convect(sem_tgv *T, int level, cudaStream_t s)
{
    sem_ctx *c = T->c;
    const bool f32 = T->op != SEM_F64 && T->op != SEM_F64_NATIVE;
    const size_t smem = conv_smem<NP>(f32);  // (a float pair has the size of a double)
    if (smem > 227 * 1024) return SEM_ERR_ARG;
    ConvArgs a;
    for (int k = 0; k < 3; ++k) {
        a.u[k] = fu(T, level, k);
        a.C[k] = fC(T, level, k);
    }
    a.s32 = stored32(T);
    a.vert = c->vert;
    a.nelx = c->nelx;
    a.nely = c->nely;
    a.E = c->E;
    const int grid = (int)(c->E < (int64_t)c->num_sms * 8 ? c->E : (int64_t)c->num_sms * 8);
    if (f32) {
        a.jinv = c->jinv32;
        a.D = c->tab32 + 2 * c->n;
        a.tab = T->tab32;
        if (T->op == SEM_F16_TC)
            return run_convect<NP, float, 1>(a, grid, smem, s);
        if (T->op == SEM_BF16_TC)
            return run_convect<NP, float, 2>(a, grid, smem, s);
        return run_convect<NP, float, 0>(a, grid, smem, s);
    }
    if (T->op == SEM_F64) {  // FP64-accurate on the FP32 pipes
        a.jinv = T->jinvdf;
        a.D = c->tabdf;
        a.tab = T->tabdf;
        return run_convect<NP, df64, 0>(a, grid, smem, s);
    }
    a.jinv = c->jinv64;
    a.D = c->tab64 + 2 * c->n;
    a.tab = T->tab64;
    return run_convect<NP, double, 0>(a, grid, smem, s);
}

// Round the FP64 values of a[0..n) to FP32 values (FP32 storage numerics).
__global__ void k_round_f32(double *__restrict__ a, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        a[t] = (double)__double2float_rn(a[t]);
}

// The pressure (the solver's iterate) stays an FP64 buffer; under FP32
// storage its values are rounded to FP32 values where it is stored.
static int round_stored(sem_tgv *T, double *a, int64_t n, cudaStream_t s)
{
    if (T->storage != SEM_F32) return SEM_OK;
    const int64_t blocks = sem_ceil_div(n, 256);
    k_round_f32<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(a, n);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

#define TGV_DISPATCH(npval, ...)            \
    switch (npval) {                        \
        SEM_NP_CASE(2, __VA_ARGS__)         \
        SEM_NP_CASE(3, __VA_ARGS__)         \
        SEM_NP_CASE(4, __VA_ARGS__)         \
        SEM_NP_CASE(5, __VA_ARGS__)         \
        SEM_NP_CASE(6, __VA_ARGS__)         \
        SEM_NP_CASE(7, __VA_ARGS__)         \
        SEM_NP_CASE(8, __VA_ARGS__)         \
        SEM_NP_CASE(9, __VA_ARGS__)         \
        SEM_NP_CASE(10, __VA_ARGS__)        \
        default: return SEM_ERR_ARG;        \
    }

static int convect(sem_tgv *T, int level, cudaStream_t s)
{
    TGV_DISPATCH(T->c->n, return launch_convect<NP>(T, level, s));
    return SEM_ERR_ARG;
}

// Move the histories between the FP64 and FP32 buffers (a change of storage
// precision between two steps; narrowing rounds to nearest).
static int move_storage(sem_tgv *T, bool to32, cudaStream_t s)
{
    const int64_t nL = T->c->nL;
    for (int l = 0; l < 3; ++l)
        for (int k = 0; k < 3; ++k) {
            if (to32) {
                k_conv_f64_f32<<<conv_grid(nL), 256, 0, s>>>(T->u[l][k], T->u32[l][k], nL);
                k_conv_f64_f32<<<conv_grid(nL), 256, 0, s>>>(T->C[l][k], T->C32[l][k], nL);
            } else {
                k_conv_f32_f64<<<conv_grid(nL), 256, 0, s>>>(T->u32[l][k], T->u[l][k], nL);
                k_conv_f32_f64<<<conv_grid(nL), 256, 0, s>>>(T->C32[l][k], T->C[l][k], nL);
            }
            SEM_CHECK_LAUNCH();
        }
    if (to32) {  // the pressure stays an FP64 buffer holding FP32 values
        k_round_f32<<<conv_grid(nL), 256, 0, s>>>(T->p, nL);
        SEM_CHECK_LAUNCH();
    }
    return SEM_OK;
}

// BDF_q / EXT_q coefficients for the step h0 = t^{n+1} - t^n after steps h1,
// h2 (Sec. 3; unequal under the CFL-controlled step).  With the distances
// s1 = h0, s2 = h0 + h1, s3 = s2 + h2 from t^{n+1} back to the earlier levels,
// differentiating and extrapolating the interpolant through those levels gives
//   q = 3: b0 = h0 (1/s1 + 1/s2 + 1/s3), b1 = s2 s3 / (h1 (h1 + h2)),
//          b2 = -h0^2 s3 / (s2 h1 h2), b3 = h0^2 s2 / (s3 (h1 + h2) h2),
//          a1 = s2 s3 / (h1 (h1 + h2)), a2 = -s1 s3 / (h1 h2), a3 = s1 s2 / ((h1 + h2) h2);
//   q = 2: b0 = h0 (1/s1 + 1/s2), b1 = s2 / h1, b2 = -h0^2 / (s2 h1),
//          a1 = s2 / h1, a2 = -s1 / h1;
//   q = 1: b0 = b1 = a1 = 1.
// Equal steps take the textbook constants exactly (11/6; 3, -3/2, 1/3; 3, -3, 1).
static Coef coef(int q, double h0, double h1, double h2)
{
    Coef k;
    memset(&k, 0, sizeof(k));
    k.dt = h0;
    const bool equal = h1 == h0 && (q < 3 || h2 == h0);
    if (q == 1) { k.b0 = 1.0; k.b[0] = 1.0; k.a[0] = 1.0; }
    else if (q == 2 && equal) { k.b0 = 1.5; k.b[0] = 2.0; k.b[1] = -0.5; k.a[0] = 2.0; k.a[1] = -1.0; }
    else if (equal) { k.b0 = 11.0 / 6.0; k.b[0] = 3.0; k.b[1] = -1.5; k.b[2] = 1.0 / 3.0; k.a[0] = 3.0; k.a[1] = -3.0; k.a[2] = 1.0; }
    else if (q == 2) {
        const double s1 = h0, s2 = h0 + h1;
        k.b0 = h0 * (1.0 / s1 + 1.0 / s2);
        k.b[0] = s2 / h1;
        k.b[1] = -h0 * h0 / (s2 * h1);
        k.a[0] = s2 / h1;
        k.a[1] = -s1 / h1;
    } else {
        const double s1 = h0, s2 = h0 + h1, s3 = s2 + h2, h12 = h1 + h2;
        k.b0 = h0 * (1.0 / s1 + 1.0 / s2 + 1.0 / s3);
        k.b[0] = s2 * s3 / (h1 * h12);
        k.b[1] = -h0 * h0 * s3 / (s2 * h1 * h2);
        k.b[2] = h0 * h0 * s2 / (s3 * h12 * h2);
        k.a[0] = s2 * s3 / (h1 * h12);
        k.a[1] = -s1 * s3 / (h1 * h2);
        k.a[2] = s1 * s2 / (h12 * h2);
    }
    return k;
}

static GapInv gap_inv(const sem_ctx *c)
{
    GapInv g;
    memset(&g, 0, sizeof(g));
    const int N = c->n - 1;
    for (int i = 0; i <= N; ++i) {
        const double l = i > 0 ? c->hxi[i] - c->hxi[i - 1] : 1e300;
        const double r = i < N ? c->hxi[i + 1] - c->hxi[i] : 1e300;
        g.v[i] = 1.0 / (l < r ? l : r);
    }
    return g;
}

static int diag(sem_tgv *T, int advance, cudaStream_t s)
{
    sem_ctx *c = T->c;
    const int blocks = (int)(c->E < 65535 * 16 ? c->E : 65535 * 16);
    // FP64-accurate on the FP32 pipes (J^-1, B and D as float pairs)
    TGV_DISPATCH(c->n, k_tgv_diag_part<NP, df64><<<blocks, 256, 0, s>>>(
                           fu(T, 0, 0), fu(T, 0, 1), fu(T, 0, 2), (int)stored32(T), T->jinvdf,
                           (const df64 *)c->geodf, (const df64 *)c->tabdf, gap_inv(c), T->part, c->E));
    SEM_CHECK_LAUNCH();
    const double V = c->volume;
    k_tgv_diag_final<<<1, 256, 0, s>>>(T->part, c->E, V, T->dt, T->dev, T->log, advance);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

static int pressure_projected(sem_tgv *T, cudaStream_t s);
static void proj_free(sem_tgv *T);

// The pressure Poisson solve A x = b (x holds the initial guess): Jacobi-PCG
// in the persistent kernel (workspace slot 4), or flexible GMRES + HSMG (its
// convergence status goes to the step's log, like the persistent solver's).
static int pressure_solve(sem_tgv *T, const double *b, double *x, int x_zero, cudaStream_t s)
{
    if (!T->psolver) return sem_pcg_solve_dev(T->c, 4, b, x, 1.0, 0.0, T->po, s);
    const int rc = sem_gmres_solve_dev(T->hsmg, 1, b, x, T->po, T->prestart, &T->pinfo, s, x_zero);
    if (rc == SEM_OK || rc == SEM_ERR_NOT_CONVERGED || rc == SEM_ERR_BREAKDOWN) return SEM_OK;
    return rc;
}

// One step of order q on stream s (capturable).
static int step_once(sem_tgv *T, int q, cudaStream_t s)
{
    sem_ctx *c = T->c;
    const int64_t nL = c->nL;
    const size_t bytes = sizeof(double) * nL;
    const Coef k = coef(q, T->dt, T->hist_dt[0], T->hist_dt[1]);
    int rc;
    const int s32 = stored32(T);
    // 1. convective term of the current velocity (stored: C history)
    rc = convect(T, 0, s);
    if (rc) return rc;
    // 2. extrapolated convection
    FArgs fa;
    for (int cc = 0; cc < 3; ++cc) {
        fa.F[cc] = T->F[cc];
        for (int l = 0; l < 3; ++l) fa.C[l][cc] = fC(T, l, cc);
    }
    fa.s32 = s32;
    k_tgv_F<<<(unsigned)sem_ceil_div(nL, 256), 256, 0, s>>>(fa, k, nL);
    SEM_CHECK_LAUNCH();
    // 3. strong right-hand side g
    GArgs ga;
    for (int cc = 0; cc < 3; ++cc) {
        ga.F[cc] = T->F[cc];
        ga.g[cc] = T->g[cc];
        for (int l = 0; l < 3; ++l) ga.u[l][cc] = fu(T, l, cc);
    }
    ga.s32 = s32;
    ga.geo64 = c->geo64;
    ga.gs = sem_gs_desc(c);
    ga.k = k;
    k_tgv_g<<<(unsigned)sem_ceil_div(c->nG, 256), 256, 0, s>>>(ga);
    SEM_CHECK_LAUNCH();
    // 4. pressure: weak divergence, dssum, Poisson solve from p^n
    const int blocks = (int)(c->E < 65535 * 16 ? c->E : 65535 * 16);
    TGV_DISPATCH(c->n, k_tgv_divg<NP, df64><<<blocks, 256, 0, s>>>(T->g[0], T->g[1], T->g[2], T->jinvdf,
                                                                   (const df64 *)c->geodf,
                                                                   (const df64 *)c->tabdf, T->bp, c->E));
    SEM_CHECK_LAUNCH();
    rc = sem_dssum_dev(c, T->bp, SEM_F64, s);
    if (rc) return rc;
    rc = T->proj_max > 0 ? pressure_projected(T, s) : pressure_solve(T, T->bp, T->p, 0, s);
    if (rc) return rc;
    rc = round_stored(T, T->p, nL, s);
    if (rc) return rc;
    int io, so;
    const char *st0 = (const char *)sem_solve_state_ptr(c, 0, &io, &so);
    const char *st1 = (const char *)sem_solve_state_ptr(c, 1, &io, &so);
    const int stride = (int)(st1 - st0);
    const int *serr = (const int *)((const char *)sem_solve_sync_ptr(c) + 8);
    if (T->psolver)
        k_tgv_log_host<<<1, 1, 0, s>>>(T->dev, T->log, 0, T->pinfo.iters, T->pinfo.status, 1);
    else
        k_tgv_log_iters<<<1, 32, 0, s>>>(st0, stride, io, so, serr, 0, 1, T->dev, T->log, 1);
    SEM_CHECK_LAUNCH();
    // 5. velocity right-hand sides and the three Helmholtz solves (from the extrapolated velocity)
    VArgs va;
    for (int cc = 0; cc < 3; ++cc) {
        va.F[cc] = T->F[cc];
        va.rhs[cc] = T->rhs[cc];
        for (int l = 0; l < 3; ++l) va.u[l][cc] = fu(T, l, cc);
    }
    va.s32 = s32;
    va.p = T->p;
    va.jinv = c->jinv64;
    va.geo64 = c->geo64;
    va.D = c->tab64 + 2 * c->n;
    va.k = k;
    va.E = c->E;
    TGV_DISPATCH(c->n, k_tgv_vrhs<NP><<<blocks, 256, 0, s>>>(va));
    SEM_CHECK_LAUNCH();
    for (int cc = 0; cc < 3; ++cc) {
        rc = sem_dssum_dev(c, T->rhs[cc], SEM_F64, s);
        if (rc) return rc;
    }
    // the solves start from the extrapolated velocity (EXT weights of the step)
    XArgs xa;
    for (int cc = 0; cc < 3; ++cc) {
        xa.x[cc] = T->unew[cc];
        for (int l = 0; l < 3; ++l) xa.u[l][cc] = fu(T, l, cc);
    }
    xa.s32 = s32;
    k_tgv_ext<<<(unsigned)sem_ceil_div(nL, 256), 256, 0, s>>>(xa, k, nL);
    SEM_CHECK_LAUNCH();
    const double *bb[3] = {T->rhs[0], T->rhs[1], T->rhs[2]};
    double *xx[3] = {T->unew[0], T->unew[1], T->unew[2]};
    // (workspace slots 5-7; slot 4 keeps the pressure's Jacobi inverse between steps)
    rc = sem_pcg_solve_dev_batch(c, 3, bb, xx, T->nu, k.b0 / T->dt, T->vo, s, 5);
    if (rc) return rc;
    k_tgv_log_iters<<<1, 32, 0, s>>>(st0, stride, io, so, serr, 1, 3, T->dev, T->log, 0);
    SEM_CHECK_LAUNCH();
    // 6. shift histories (copies keep every buffer address fixed for graph replay)
    const size_t sbytes = (s32 ? sizeof(float) : sizeof(double)) * nL;
    for (int cc = 0; cc < 3; ++cc) {
        SEM_CUDA(cudaMemcpyAsync(fu(T, 2, cc), fu(T, 1, cc), sbytes, cudaMemcpyDeviceToDevice, s));
        SEM_CUDA(cudaMemcpyAsync(fu(T, 1, cc), fu(T, 0, cc), sbytes, cudaMemcpyDeviceToDevice, s));
        if (s32) {  // the new velocity, rounded to FP32 where it is stored
            k_conv_f64_f32<<<conv_grid(nL), 256, 0, s>>>(T->unew[cc], T->u32[0][cc], nL);
            SEM_CHECK_LAUNCH();
        } else {
            SEM_CUDA(cudaMemcpyAsync(T->u[0][cc], T->unew[cc], bytes, cudaMemcpyDeviceToDevice, s));
        }
        SEM_CUDA(cudaMemcpyAsync(fC(T, 2, cc), fC(T, 1, cc), sbytes, cudaMemcpyDeviceToDevice, s));
        SEM_CUDA(cudaMemcpyAsync(fC(T, 1, cc), fC(T, 0, cc), sbytes, cudaMemcpyDeviceToDevice, s));
    }
    return diag(T, 1, s);
}

extern "C" void sem_tgv_destroy(sem_tgv *T)
{
    if (!T) return;
    cudaDeviceSynchronize();
    if (T->graph_state == 1) cudaGraphExecDestroy(T->graph);
    proj_free(T);
    if (T->block) cudaFree(T->block);
    if (T->block32) cudaFree(T->block32);
    if (T->part) cudaFree(T->part);
    if (T->tab64) cudaFree(T->tab64);
    if (T->tab32) cudaFree(T->tab32);
    if (T->tabdf) cudaFree(T->tabdf);
    if (T->jinvdf) cudaFree(T->jinvdf);
    if (T->log) cudaFree(T->log);
    if (T->dev) cudaFree(T->dev);
    if (T->hlog) cudaFreeHost(T->hlog);
    if (T->hdev) cudaFreeHost(T->hdev);
    sem_hsmg_destroy(T->hsmg);
    free(T);
}

extern "C" int sem_tgv_init(sem_ctx *c, double nu, double dt, sem_dtype op, const sem_solve_opts *vel,
                            const sem_solve_opts *pres, sem_tgv **out)
{
    if (!out) return SEM_ERR_ARG;
    *out = nullptr;
    if (!c || !(nu > 0) || !(dt > 0) || (op != SEM_F64 && op != SEM_F32 && op != SEM_F64_NATIVE))
        return SEM_ERR_ARG;
    if (!c->periodic[0] || !c->periodic[1] || !c->periodic[2] || c->n > 10) return SEM_ERR_ARG;
    sem_tgv *T = (sem_tgv *)calloc(1, sizeof(sem_tgv));
    if (!T) return SEM_ERR_NOMEM;
    T->c = c;
    T->nu = nu;
    T->dt = dt;
    T->hist_dt[0] = T->hist_dt[1] = dt;
    T->op = op;
    sem_solve_opts_default(&T->vo);
    sem_solve_opts_default(&T->po);
    if (vel) T->vo = *vel;
    if (pres) T->po = *pres;
    if (op == SEM_F32 && !pres) T->po.inner = SEM_F32;
    T->storage = SEM_F64;
    T->op0 = op;
    T->vin0 = T->vo.inner;
    T->pin0 = T->po.inner;
    T->cur_rule = -1;
    const int n = c->n;
    T->M = (3 * n + 1) / 2;
    const int64_t nL = c->nL;
#define TGV_TRY(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            sem_note_cuda_error(e_, #call);                                                  \
            sem_tgv_destroy(T);                                                              \
            return e_ == cudaErrorMemoryAllocation ? SEM_ERR_NOMEM : SEM_ERR_CUDA;           \
        }                                                                                    \
    } while (0)
    // fields: u 9, C 9, p 1, unew 3, F 3, g 3, bp 1, rhs 3 = 32 E-vectors
    TGV_TRY(cudaMalloc(&T->block, sizeof(double) * 32 * nL));
    TGV_TRY(cudaMemset(T->block, 0, sizeof(double) * 32 * nL));
    double *b = T->block;
    for (int l = 0; l < 3; ++l)
        for (int k = 0; k < 3; ++k) { T->u[l][k] = b; b += nL; }
    for (int l = 0; l < 3; ++l)
        for (int k = 0; k < 3; ++k) { T->C[l][k] = b; b += nL; }
    T->p = b; b += nL;
    for (int k = 0; k < 3; ++k) { T->unew[k] = b; b += nL; }
    for (int k = 0; k < 3; ++k) { T->F[k] = b; b += nL; }
    for (int k = 0; k < 3; ++k) { T->g[k] = b; b += nL; }
    T->bp = b; b += nL;
    for (int k = 0; k < 3; ++k) { T->rhs[k] = b; b += nL; }
    TGV_TRY(cudaMalloc(&T->part, sizeof(double) * 3 * c->E));
    // dealiasing tables
    double eta[64], wq[64], J[64 * SEM_NPMAX], h64[2 * 64 + 64 * SEM_NPMAX];
    float h32[2 * 64 + 64 * SEM_NPMAX];
    gl_table(T->M, eta, wq);
    interp_table(n, c->hxi, T->M, eta, J);
    const int ntab = 2 * T->M + T->M * n;
    for (int q = 0; q < T->M; ++q) { h64[q] = eta[q]; h64[T->M + q] = wq[q]; }
    for (int t = 0; t < T->M * n; ++t) h64[2 * T->M + t] = J[t];
    for (int t = 0; t < ntab; ++t) h32[t] = (float)h64[t];
    TGV_TRY(cudaMalloc(&T->tab64, sizeof(double) * ntab));
    TGV_TRY(cudaMalloc(&T->tab32, sizeof(float) * ntab));
    TGV_TRY(cudaMemcpy(T->tab64, h64, sizeof(double) * ntab, cudaMemcpyHostToDevice));
    TGV_TRY(cudaMemcpy(T->tab32, h32, sizeof(float) * ntab, cudaMemcpyHostToDevice));
    {
        df64 hdf[2 * 64 + 64 * SEM_NPMAX];
        for (int t = 0; t < ntab; ++t) {
            const float h = (float)h64[t];
            hdf[t] = df64(h, (float)(h64[t] - (double)h));
        }
        TGV_TRY(cudaMalloc(&T->tabdf, sizeof(df64) * ntab));
        TGV_TRY(cudaMemcpy(T->tabdf, hdf, sizeof(df64) * ntab, cudaMemcpyHostToDevice));
    }
    TGV_TRY(cudaMalloc(&T->log, sizeof(TgvLogEntry) * TGV_LOG));
    TGV_TRY(cudaMemset(T->log, 0, sizeof(TgvLogEntry) * TGV_LOG));
    TGV_TRY(cudaMallocHost(&T->hlog, sizeof(TgvLogEntry) * TGV_LOG));
    TGV_TRY(cudaMallocHost(&T->hdev, sizeof(TgvDev)));
    TGV_TRY(cudaMalloc(&T->dev, sizeof(TgvDev)));
    TGV_TRY(cudaMemset(T->dev, 0, sizeof(TgvDev)));
    // J^{-1} on the context and three solver workspaces for the velocity batch
    if (!c->jinv64) {
        TGV_TRY(cudaMalloc(&c->jinv64, sizeof(double) * 9 * nL));
        TGV_TRY(cudaMalloc(&c->jinv32, sizeof(float) * 9 * nL));
        int rc = sem_run_geometry(c, nullptr, true, 0);
        if (rc) { sem_tgv_destroy(T); return rc; }
    }
    TGV_TRY(cudaMalloc(&T->jinvdf, sizeof(df64) * 9 * nL));
    k_split_df64<<<(unsigned)sem_ceil_div(9 * nL, 256), 256>>>(c->jinv64, T->jinvdf, 9 * nL);
    TGV_TRY(cudaGetLastError());
    for (int slot = 4; slot < 8; ++slot) {  // the stepper's own solver workspaces
        if (c->ws[slot].r) continue;
        int rc = sem_alloc_ws(c, slot);
        if (rc) { sem_tgv_destroy(T); return rc; }
    }
    TGV_TRY(cudaDeviceSynchronize());
#undef TGV_TRY
    *out = T;
    return SEM_OK;
}

static int stage_field(sem_ctx *c, const double *src, double *dst, cudaStream_t s)
{
    const size_t bytes = sizeof(double) * c->nL;
    const cudaMemcpyKind kind = sem_is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SEM_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
    return SEM_OK;
}

__global__ void k_tgv_set_time(TgvDev *dv, double t) { dv->t = t; }

extern "C" int sem_tgv_set(sem_tgv *T, int level, const double *u, const double *v, const double *w,
                           const double *p, int step, double t, void *stream)
{
    if (!T || level < 0 || level > 2 || !u || !v || !w || step < 0) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const double *src[3] = {u, v, w};
    for (int k = 0; k < 3; ++k) {
        int rc = stage_field(T->c, src[k], T->u[level][k], s);
        if (rc) return rc;
        if (stored32(T)) {
            k_conv_f64_f32<<<conv_grid(T->c->nL), 256, 0, s>>>(T->u[level][k], T->u32[level][k], T->c->nL);
            SEM_CHECK_LAUNCH();
        }
    }
    if (level == 0 && p) {
        int rc = stage_field(T->c, p, T->p, s);
        if (rc) return rc;
    }
    if (level > 0) {  // history of the convective term at that level
        int rc = convect(T, level, s);
        if (rc) return rc;
    }
    if (level == 0) {
        T->step = step;
        T->t = t;
        T->hist_dt[0] = T->hist_dt[1] = T->dt;  // earlier levels: steps of the current size
        k_tgv_set_time<<<1, 1, 0, s>>>(T->dev, t);
        SEM_CHECK_LAUNCH();
    }
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
}

// ---------------------------------------------------------------------------
// Projection of the pressure solve onto previous solutions (Sec. 3: the
// pressure solver keeps a projection space of dimension 20).  This is the
// A-conjugate projection of Fischer (1998): with an A-orthonormal basis X of
// earlier solutions and BX = A X,
//     alpha = X^T b,  x_bar = X alpha,  b' = b - BX alpha,
// the solve is for the remainder A dx = b', p = x_bar + dx, and dx (A-
// orthogonalised twice against X, classical Gram-Schmidt, then A-normalised)
// joins the basis; a full basis restarts from the latest solution p.  Inner
// products are the assembled ones (local sums weighted by 1/multiplicity).
// Everything stays on the device, so a captured step replays it.
// ---------------------------------------------------------------------------

#define TGV_PMAX 32   // largest basis
#define TGV_PBLK 304  // blocks of the dot kernels (fixed: deterministic sums)

// part[b][k] = block b's share of sum_i X_k[i] v[i] w[i], k < L (L = *Ld): the
// basis is swept in chunks of TGV_PCH vectors, each with its accumulators in
// registers (v and w are read once per chunk).
#define TGV_PCH 8
__global__ void __launch_bounds__(256, 2) k_proj_dot(const double *__restrict__ X, const double *__restrict__ v,
                                                     const double *__restrict__ w, const int *__restrict__ Ld,
                                                     int64_t n, double *__restrict__ part)
{
    __shared__ double red[8][TGV_PCH];
    const int L = *Ld;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int k0 = 0; k0 < L; k0 += TGV_PCH) {
        const int m = L - k0 < TGV_PCH ? L - k0 : TGV_PCH;
        double acc[TGV_PCH];
#pragma unroll
        for (int k = 0; k < TGV_PCH; ++k) acc[k] = 0.0;
        const double *Xc = X + (int64_t)k0 * n;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double t = v[i] * w[i];
#pragma unroll
            for (int k = 0; k < TGV_PCH; ++k)
                if (k < m) acc[k] = fma(__ldcg(Xc + (int64_t)k * n + i), t, acc[k]);
        }
#pragma unroll
        for (int k = 0; k < TGV_PCH; ++k) {
            double a = acc[k];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[wp][k] = a;
        }
        __syncthreads();
        if (threadIdx.x < m) {
            double a = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += red[q][threadIdx.x];
            part[(int64_t)blockIdx.x * TGV_PMAX + k0 + threadIdx.x] = a;
        }
        __syncthreads();
    }
}

// c[k] = sum over blocks of part[b][k] in block order, k < L.
__global__ void k_proj_dot_final(const double *__restrict__ part, const int *__restrict__ Ld,
                                 double *__restrict__ c)
{
    const int L = *Ld, lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < L; k += blockDim.x >> 5) {
        double a = 0.0;
        for (int b = lane; b < TGV_PBLK; b += 32) a += part[(int64_t)b * TGV_PMAX + k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) c[k] = a;
    }
}

// out[i] = (a ? a[i] : 0) + sg * sum_{k<L} c[k] X_k[i]  (out may alias a).
__global__ void k_proj_axpy(double *out, const double *a, const double *__restrict__ X,
                            const double *__restrict__ c, double sg, const int *__restrict__ Ld, int64_t n)
{
    const int L = *Ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < L; ++k) s = fma(c[k], __ldcg(X + (int64_t)k * n + i), s);
        out[i] = fma(sg, s, a ? a[i] : 0.0);
    }
}

__global__ void k_vec_add(double *out, const double *a, const double *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// Before the update: a full basis restarts (L = 0) and the latest solution p
// replaces dx as the vector to add.  pint = {L, 1, restart}.
__global__ void k_proj_restart(int *pint, int Lmax)
{
    pint[2] = pint[0] >= Lmax;
    if (pint[2]) pint[0] = 0;
}

__global__ void k_copy_if(double *dst, const double *src, const int *flag, int64_t n)
{
    if (!*flag) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Append v / |v|_A and A v / |v|_A as basis vector L when the A-norm left after
// the orthogonalisation is not round-off (nrm[1] > 1e-20 nrm[0], nrm[0] = the
// A-norm squared before it).  The count is raised by k_proj_inc afterwards.
__global__ void k_proj_append(double *X, double *BX, const double *v, const double *av,
                              const double *nrm, const int *pint, int64_t n)
{
    const double n0 = nrm[0], n1 = nrm[1];
    if (!(n1 > 1e-20 * n0) || !(n1 > 0.0)) return;
    const int L = pint[0];
    const double s = 1.0 / sqrt(n1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        X[(int64_t)L * n + i] = v[i] * s;
        BX[(int64_t)L * n + i] = av[i] * s;
    }
}

__global__ void k_proj_inc(int *pint, const double *nrm)
{
    if (nrm[1] > 1e-20 * nrm[0] && nrm[1] > 0.0) pint[0] += 1;
}

__global__ void k_recip_inplace(double *a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 1.0 / a[i];
}

__global__ void k_fill(double *a, double v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

static unsigned vec_grid(int64_t n)
{
    const int64_t b = sem_ceil_div(n, 256);
    return (unsigned)(b < 2048 ? b : 2048);
}

// c[0..L) = <X_k, v> (assembled), L from *Ld.
static int proj_dot(sem_tgv *T, const double *X, const double *v, const int *Ld, double *c, cudaStream_t s)
{
    const int64_t n = T->c->nL;
    k_proj_dot<<<TGV_PBLK, 256, 0, s>>>(X, v, T->pw, Ld, n, T->ppart);
    SEM_CHECK_LAUNCH();
    k_proj_dot_final<<<1, 1024, 0, s>>>(T->ppart, Ld, c);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

static void proj_free(sem_tgv *T)
{
    double *ps[] = {T->pX, T->pBX, T->pw, T->pxb, T->pbq, T->pdx, T->padx, T->pcoef, T->ppart};
    for (double *p : ps)
        if (p) cudaFree(p);
    if (T->pint) cudaFree(T->pint);
    T->pX = T->pBX = T->pw = T->pxb = T->pbq = T->pdx = T->padx = T->pcoef = T->ppart = nullptr;
    T->pint = nullptr;
    T->proj_max = 0;
}

// The pressure solve of one step with projection (capturable): p from bp.
static int pressure_projected(sem_tgv *T, cudaStream_t s)
{
    sem_ctx *c = T->c;
    const int64_t n = c->nL;
    const unsigned g = vec_grid(n);
    int *L = T->pint, *one = T->pint + 1, *restart = T->pint + 2;
    double *alpha = T->pcoef, *nrm = T->pcoef + TGV_PMAX;
    int rc;
    // projection of the new right-hand side
    if ((rc = proj_dot(T, T->pX, T->bp, L, alpha, s))) return rc;
    k_proj_axpy<<<g, 256, 0, s>>>(T->pxb, nullptr, T->pX, alpha, 1.0, L, n);
    k_proj_axpy<<<g, 256, 0, s>>>(T->pbq, T->bp, T->pBX, alpha, -1.0, L, n);
    SEM_CHECK_LAUNCH();
    // the remainder, from a zero guess
    SEM_CUDA(cudaMemsetAsync(T->pdx, 0, sizeof(double) * n, s));
    if ((rc = pressure_solve(T, T->pbq, T->pdx, 1, s))) return rc;
    k_vec_add<<<g, 256, 0, s>>>(T->p, T->pxb, T->pdx, n);
    SEM_CHECK_LAUNCH();
    // basis update: v = dx (or p after a restart), A v, CGS twice, A-normalise, append
    k_proj_restart<<<1, 1, 0, s>>>(T->pint, T->proj_max);
    k_copy_if<<<g, 256, 0, s>>>(T->pdx, T->p, restart, n);
    SEM_CHECK_LAUNCH();
    if ((rc = sem_ax_dev(c, T->pdx, T->padx, 1.0, 0.0, SEM_F64, s))) return rc;
    if ((rc = sem_dssum_dev(c, T->padx, SEM_F64, s))) return rc;
    k_proj_dot<<<TGV_PBLK, 256, 0, s>>>(T->pdx, T->padx, T->pw, one, n, T->ppart);
    k_proj_dot_final<<<1, 1024, 0, s>>>(T->ppart, one, nrm);
    SEM_CHECK_LAUNCH();
    for (int pass = 0; pass < 2; ++pass) {
        if ((rc = proj_dot(T, T->pBX, T->pdx, L, alpha, s))) return rc;
        k_proj_axpy<<<g, 256, 0, s>>>(T->pdx, T->pdx, T->pX, alpha, -1.0, L, n);
        k_proj_axpy<<<g, 256, 0, s>>>(T->padx, T->padx, T->pBX, alpha, -1.0, L, n);
        SEM_CHECK_LAUNCH();
    }
    k_proj_dot<<<TGV_PBLK, 256, 0, s>>>(T->pdx, T->padx, T->pw, one, n, T->ppart);
    k_proj_dot_final<<<1, 1024, 0, s>>>(T->ppart, one, nrm + 1);
    k_proj_append<<<g, 256, 0, s>>>(T->pX, T->pBX, T->pdx, T->padx, nrm, T->pint, n);
    k_proj_inc<<<1, 1, 0, s>>>(T->pint, nrm);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

extern "C" int sem_tgv_set_projection(sem_tgv *T, int max_vectors)
{
    if (!T || max_vectors < 0 || max_vectors > TGV_PMAX) return SEM_ERR_ARG;
    SEM_CUDA(cudaDeviceSynchronize());
    proj_free(T);
    if (T->graph_state == 1) {
        cudaGraphExecDestroy(T->graph);
        T->graph_state = 0;
        T->graph_warm = 0;
    }
    if (max_vectors == 0) return SEM_OK;
    sem_ctx *c = T->c;
    const int64_t n = c->nL;
    const size_t vb = sizeof(double) * (size_t)n;
    bool ok = cudaMalloc(&T->pX, vb * max_vectors) == cudaSuccess &&
              cudaMalloc(&T->pBX, vb * max_vectors) == cudaSuccess &&
              cudaMalloc(&T->pw, vb) == cudaSuccess && cudaMalloc(&T->pxb, vb) == cudaSuccess &&
              cudaMalloc(&T->pbq, vb) == cudaSuccess && cudaMalloc(&T->pdx, vb) == cudaSuccess &&
              cudaMalloc(&T->padx, vb) == cudaSuccess &&
              cudaMalloc(&T->pcoef, sizeof(double) * (TGV_PMAX + 2)) == cudaSuccess &&
              cudaMalloc(&T->ppart, sizeof(double) * TGV_PBLK * TGV_PMAX) == cudaSuccess &&
              cudaMalloc(&T->pint, sizeof(int) * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        proj_free(T);
        return SEM_ERR_NOMEM;
    }
    const int h[4] = {0, 1, 0, 0};
    SEM_CUDA(cudaMemcpy(T->pint, h, sizeof(h), cudaMemcpyHostToDevice));
    // weights 1/multiplicity: dssum of ones
    k_fill<<<vec_grid(n), 256>>>(T->pw, 1.0, n);
    SEM_CHECK_LAUNCH();
    int rc = sem_dssum_dev(c, T->pw, SEM_F64, 0);
    if (rc) return rc;
    k_recip_inplace<<<vec_grid(n), 256>>>(T->pw, n);
    SEM_CHECK_LAUNCH();
    SEM_CUDA(cudaDeviceSynchronize());
    T->proj_max = max_vectors;
    return SEM_OK;
}

static bool conv_dtype_ok(sem_dtype d)
{
    return d == SEM_F64 || d == SEM_F64_NATIVE || d == SEM_F32 || d == SEM_F16_TC || d == SEM_BF16_TC;
}

static bool solve_dtype_ok(sem_dtype d)
{
    return d == SEM_F64 || d == SEM_F64_NATIVE || d == SEM_F32 || d == SEM_F16_TC || d == SEM_BF16_TC;
}

extern "C" int sem_tgv_set_policy(sem_tgv *T, int n, const sem_tgv_policy *rules)
{
    if (!T || n < 0 || n > SEM_TGV_MAX_RULES || (n > 0 && !rules)) return SEM_ERR_ARG;
    for (int r = 0; r < n; ++r) {
        const sem_tgv_policy &p = rules[r];
        if (!conv_dtype_ok(p.sem) || !solve_dtype_ok(p.vel) || !solve_dtype_ok(p.pres) ||
            (p.storage != SEM_F64 && p.storage != SEM_F32))
            return SEM_ERR_ARG;
        if (r > 0 && p.first_step < rules[r - 1].first_step) return SEM_ERR_ARG;
    }
    bool need32 = false;
    for (int r = 0; r < n; ++r) need32 |= rules[r].storage == SEM_F32;
    if (need32 && !T->block32) {  // FP32 history buffers: 18 FP32 E-vectors
        const int64_t nL = T->c->nL;
        cudaError_t e = cudaMalloc(&T->block32, sizeof(float) * 18 * nL);
        if (e != cudaSuccess) {
            sem_note_cuda_error(e, "cudaMalloc(FP32 histories)");
            T->block32 = nullptr;
            return e == cudaErrorMemoryAllocation ? SEM_ERR_NOMEM : SEM_ERR_CUDA;
        }
        float *b = T->block32;
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) { T->u32[l][k] = b; b += nL; }
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k) { T->C32[l][k] = b; b += nL; }
    }
    for (int r = 0; r < n; ++r) T->rules[r] = rules[r];
    T->nrules = n;
    T->cur_rule = -2;  // re-applied before the next step
    return SEM_OK;
}

// Put the rule in force at step `step` (1-based) into effect; a change drops
// the captured step graph so that the next steady step is captured again, and
// a change of storage precision moves the histories to the other buffers.
static int apply_policy(sem_tgv *T, int step, cudaStream_t s)
{
    int r = -1;
    for (int k = 0; k < T->nrules; ++k)
        if (T->rules[k].first_step <= step) r = k;
    if (r == T->cur_rule) return SEM_OK;
    const bool was32 = stored32(T);
    if (r < 0) {
        T->op = T->op0;
        T->vo.inner = T->vin0;
        T->po.inner = T->pin0;
        T->storage = SEM_F64;
    } else {
        T->op = T->rules[r].sem;
        T->vo.inner = T->rules[r].vel;
        T->po.inner = T->rules[r].pres;
        T->storage = T->rules[r].storage;
    }
    if (T->graph_state == 1) {
        cudaGraphExecDestroy(T->graph);
        T->graph_state = 0;
    }
    T->graph_warm = 0;
    T->cur_rule = r;
    if (was32 != stored32(T)) return move_storage(T, stored32(T), s);
    return SEM_OK;
}

// Advance nsteps steps on stream s (no synchronisation).
static int advance(sem_tgv *T, int nsteps, cudaStream_t s)
{
    for (int it = 0; it < nsteps; ++it) {
        const int q = T->step + 1 < 3 ? T->step + 1 : 3;
        const bool adaptive = T->cfl_target > 0;
        // graph replay only for third-order steps of one fixed size (and a
        // pressure solver that does not read back to the host)
        const bool steady = q == 3 && !adaptive && !T->psolver && T->hist_dt[0] == T->dt &&
                            T->hist_dt[1] == T->dt;
        int rc = apply_policy(T, T->step + 1, s);
        if (rc) return rc;
        if (steady && s != 0 && T->graph_state == 0 && !T->graph_warm) {
            // one steady step runs directly first, so the Jacobi inverses of its
            // solves are cached when the next one is captured (the graph then
            // keeps reusing them)
            T->graph_warm = 1;
        } else if (steady && s != 0 && T->graph_state == 0) {
            // capture one steady-state step; fall back to direct launches if capture fails
            cudaGraph_t g = nullptr;
            T->graph_state = -1;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                rc = step_once(T, 3, s);
                cudaError_t ce = cudaStreamEndCapture(s, &g);
                if (rc == SEM_OK && ce == cudaSuccess && g &&
                    cudaGraphInstantiate(&T->graph, g, 0) == cudaSuccess) {
                    T->graph_state = 1;
                    T->graph_stream = s;
                }
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
        }
        if (steady && T->graph_state == 1) {
            SEM_CUDA(cudaGraphLaunch(T->graph, s));
        } else {
            rc = step_once(T, q, s);
            if (rc) return rc;
        }
        T->step += 1;
        T->t += T->dt;
        T->hist_dt[1] = T->hist_dt[0];
        T->hist_dt[0] = T->dt;
        if (adaptive) {
            // next step from this step's CFL number: towards the target, by at
            // most +10 % and -50 % a step, capped by dt_max (a zero or NaN CFL
            // keeps the step)
            SEM_CUDA(cudaMemcpyAsync(T->hdev, T->dev, sizeof(TgvDev), cudaMemcpyDeviceToHost, s));
            SEM_CUDA(cudaStreamSynchronize(s));
            const double cfl = T->hdev->cfl;
            if (cfl > 0) {
                double f = T->cfl_target / cfl;
                if (f > 1.1) f = 1.1;
                if (f < 0.5) f = 0.5;
                T->dt = T->dt * f;
                if (T->dt_max > 0 && T->dt > T->dt_max) T->dt = T->dt_max;
            }
        }
    }
    return SEM_OK;
}

extern "C" int sem_tgv_set_pressure_solver(sem_tgv *T, int kind, int restart, sem_dtype vcycle)
{
    if (!T || kind < 0 || kind > 1) return SEM_ERR_ARG;
    if (kind == 1 && (restart < 1 || restart > 64 || (vcycle != SEM_F32 && vcycle != SEM_F64))) return SEM_ERR_ARG;
    if (T->graph_state == 1) {
        cudaGraphExecDestroy(T->graph);
        T->graph_state = 0;
    }
    T->graph_warm = 0;
    SEM_CUDA(cudaDeviceSynchronize());
    sem_hsmg_destroy(T->hsmg);
    T->hsmg = nullptr;
    T->psolver = 0;
    if (kind == 0) return SEM_OK;
    // levels N, 3, 1 (N, 2, 1 for N = 3 or 4; N, 1 below)
    const int N = T->c->N;
    int orders[3] = {N, N >= 5 ? 3 : 2, 1}, nlev = N >= 3 ? 3 : (N == 2 ? 2 : 1);
    if (nlev == 2) orders[1] = 1;
    int rc = sem_hsmg_create(T->c, nlev, orders, 1.0, 0.0, vcycle, 0.1, 200, &T->hsmg);
    if (rc) return rc;
    T->psolver = 1;
    T->prestart = restart;
    return SEM_OK;
}

extern "C" int sem_tgv_set_dt(sem_tgv *T, double dt, double cfl_target, double dt_max)
{
    if (!T || !(dt >= 0) || !(cfl_target >= 0) || !(dt_max >= 0)) return SEM_ERR_ARG;
    if (dt > 0) T->dt = dt;
    T->cfl_target = cfl_target;
    T->dt_max = dt_max;
    if (T->graph_state == 1 && (dt > 0 || cfl_target > 0)) {  // the graph holds the old step's coefficients
        cudaGraphExecDestroy(T->graph);
        T->graph_state = 0;
    }
    if (dt > 0 || cfl_target > 0) T->graph_warm = 0;
    return SEM_OK;
}

extern "C" int sem_tgv_step(sem_tgv *T, int nsteps, sem_tgv_diag *out, void *stream)
{
    if (!T || nsteps < 0) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!out) return advance(T, nsteps, s);
    // the device log is a ring of TGV_LOG entries: read it back after every
    // TGV_LOG steps at most
    int worst = SEM_OK;
    for (int done = 0; done < nsteps;) {
        const int n = nsteps - done < TGV_LOG ? nsteps - done : TGV_LOG;
        SEM_CUDA(cudaMemcpyAsync(&T->hlog[0], T->dev, sizeof(TgvDev), cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
        const long long first = ((TgvDev *)&T->hlog[0])->count;
        const int rc = advance(T, n, s);
        if (rc) return rc;
        SEM_CUDA(cudaMemcpyAsync(T->hlog, T->log, sizeof(TgvLogEntry) * TGV_LOG, cudaMemcpyDeviceToHost, s));
        SEM_CUDA(cudaStreamSynchronize(s));
        for (int it = 0; it < n; ++it) {
            const TgvLogEntry &L = T->hlog[(first + it) % TGV_LOG];
            sem_tgv_diag &D = out[done + it];
            D.t = L.t;
            D.ke = L.ke;
            D.enstrophy = L.en;
            for (int k = 0; k < 4; ++k) D.iters[k] = L.iters[k];
            D.status = L.status;
            D.dt = L.dt;
            D.cfl = L.cfl;
            if (L.status != 0 && worst == SEM_OK) worst = L.status;
        }
        done += n;
    }
    return worst;
}

extern "C" int sem_tgv_get(sem_tgv *T, double *u, double *v, double *w, double *p, void *stream)
{
    if (!T) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * T->c->nL;
    double *dst[4] = {u, v, w, p};
    const double *src[4] = {T->u[0][0], T->u[0][1], T->u[0][2], T->p};
    for (int k = 0; k < 4; ++k) {
        if (!dst[k]) continue;
        if (k < 3 && stored32(T)) {  // widened through the (between steps unused) new-velocity buffer
            k_conv_f32_f64<<<conv_grid(T->c->nL), 256, 0, s>>>(T->u32[0][k], T->unew[k], T->c->nL);
            SEM_CHECK_LAUNCH();
            src[k] = T->unew[k];
        }
        const cudaMemcpyKind kind = sem_is_device_ptr(dst[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        SEM_CUDA(cudaMemcpyAsync(dst[k], src[k], bytes, kind, s));
    }
    SEM_CUDA(cudaStreamSynchronize(s));
    return SEM_OK;
}

extern "C" int sem_tgv_energy(sem_tgv *T, double *ke, double *en, void *stream)
{
    if (!T || !ke || !en) return SEM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = diag(T, 0, s);
    if (rc) return rc;
    TgvDev h;
    SEM_CUDA(cudaMemcpyAsync(&h, T->dev, sizeof(TgvDev), cudaMemcpyDeviceToHost, s));
    SEM_CUDA(cudaStreamSynchronize(s));
    TgvLogEntry L;
    SEM_CUDA(cudaMemcpy(&L, T->log + (h.count % TGV_LOG), sizeof(L), cudaMemcpyDeviceToHost));
    *ke = L.ke;
    *en = L.en;
    return SEM_OK;
}
