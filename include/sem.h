/*
 * sem.h -- C ABI of libsem: the GB300 (sm_103a) spectral-element hot path.
 *
 * The operations are those of a matrix-free SEM Navier-Stokes solver in the
 * P_N-P_N splitting (Chen, Muensch, Iakymchuk, "Mixed-Precision SEM-Based CFD
 * Simulations on GPUs: A Taylor-Green Vortex case"): the Helmholtz operator
 * ax_helm (Sec. 4, Table 2 rows B-6/B-7), the gather-scatter direct-stiffness
 * sum (Sec. 2, "gather/scatter" in the other-operations block), the Jacobi
 * preconditioned CG of the velocity solve with higher-precision reductions
 * (Sec. 1.1; Sec. 2, reductions capped at fp64), and the Taylor-Green vortex
 * time step with dealiased advection (Sec. 3; Sec. 1.1 Fig. 3 hotspots).
 * The paper prints no SEM formula; the operators are the textbook ones
 * (Deville, Fischer & Mund 2002) restated in each declaration below.
 *
 * Conventions for every entry point:
 *  - Field arguments are E-vectors: E*(N+1)^3 contiguous values, layout
 *    [E][N+1][N+1][N+1] with i (the r direction) fastest and element
 *    e = ex + nelx*(ey + nely*ez).  Their element type follows the sem_dtype
 *    argument: double for SEM_F64, float for the other three.
 *  - Field pointers may be device memory (the fast path) or host memory
 *    (pinned or pageable); host buffers are staged through device buffers
 *    owned by the context, allocated on the first such call (sem_ax also
 *    creates two streams and a few events then, and overlaps the copies of
 *    its element chunks with the operator on the other chunks).  Exception:
 *    sem_ax with SEM_F64 on pinned host buffers runs the operator on the
 *    mapped host memory itself (the kernel's loads and stores cross the host
 *    link; no staging).  Host-pointer calls return after the result is in
 *    place.
 *  - The caller owns every field buffer.  The library owns the geometry and
 *    the solver workspaces; it allocates only in sem_setup, sem_tgv_init and
 *    the first host-pointer call, never inside a device-pointer hot call.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream);
 *    device-pointer calls are asynchronous and stream ordered.
 *  - Every int-returning call returns SEM_OK (0) or a negative SEM_ERR_*.
 *    No call aborts, traps or throws across the ABI.
 *  - One context may be used by one host thread at a time.
 *  - Supported polynomial orders: 1 <= N <= 15.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SEM_API __attribute__((visibility("default")))
#else
#define SEM_API
#endif

#define SEM_OK 0
#define SEM_ERR_ARG (-1)           /* invalid argument (size, order, pointer, dtype) */
#define SEM_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define SEM_ERR_NOMEM (-3)         /* device or host allocation failed */
#define SEM_ERR_BAD_MESH (-4)      /* a non-positive Jacobian determinant */
#define SEM_ERR_NOT_CONVERGED (-5) /* maxit reached; x holds the last iterate */
#define SEM_ERR_BREAKDOWN (-6)     /* <p,Ap> <= 0 or a non-finite residual */
#define SEM_ERR_TIMEOUT (-7)       /* a bounded device-side wait gave up */
#define SEM_ERR_TOO_LARGE (-8)     /* problem larger than a fixed-size scratch area */

typedef enum {
    SEM_F64 = 0,       /* FP64 storage, FP64-accurate arithmetic (see below) */
    SEM_F32 = 1,       /* FP32 storage and arithmetic */
    SEM_BF16_TC = 2,   /* FP32 storage, BF16 tensor-core contractions, FP32 accumulation */
    SEM_F16_TC = 3,    /* FP32 storage, FP16 tensor-core contractions, FP32 accumulation */
    SEM_F64_NATIVE = 4, /* FP64 storage, native FP64 FMA arithmetic */
    SEM_F16X2_TC = 5,   /* FP32 storage, FP16 tensor-core contractions of split operands */
    SEM_BF16X3_TC = 6,  /* FP32 storage, BF16 tensor-core contractions of split operands */
    SEM_F32_TUNED = 7   /* (solver inner operator only) the FP32-accurate inner path chosen per order
                           by sem_tune_inner; see there */
} sem_dtype;
/* SEM_F16X2_TC / SEM_BF16X3_TC (N <= 7): every contracted value and D are
 * split into two FP16 (three BF16) parts, and the tensor cores sum the part
 * products that carry FP32-level accuracy (about 2^-22) with FP32
 * accumulation; FP16 parts of an element are first scaled by a power of two
 * into FP16's range.  As inner operators of refinement they converge where
 * the plain 16-bit operators (whose error relative to the smallest modes is
 * the condition number times 2^-8 or 2^-11) do not. */
/* SEM_F64 in sem_ax evaluates the FP64 operator on the FP32 pipes with
 * error-free transformations (per-element block-floating-point pairs with
 * exact folds and fused exact-product accumulation for odd N <= 11, float
 * pairs with compensated sums otherwise; per-element power-of-two scaling);
 * it meets the same FP64 accuracy bar as SEM_F64_NATIVE (max error <= 1e-12
 * of the largest output) and is several times faster on parts whose FP64
 * rate is a small fraction of their FP32 rate. */

typedef struct sem_ctx sem_ctx;
typedef struct sem_tgv sem_tgv;

typedef struct {
    int N, nelx, nely, nelz;
    int periodic[3];
    int64_t E;      /* elements */
    int64_t nL;     /* local (element-duplicated) nodes = E (N+1)^3 */
    int64_t nG;     /* unique nodes */
    double volume;  /* sum of the local mass B */
} sem_ctx_info;

/* Build a context on the current CUDA device (Sec. 1.1 Fig. 3, pre-processing).
 * N: polynomial order, 1..15.  nelx, nely, nelz >= 1 elements per direction.
 * extents: box lengths (host, 3 doubles; origin at 0) used when vertices is
 * NULL.  periodic: 3 flags (host).  vertices: NULL for a uniform box, else a
 * host array of (nelz+1)(nely+1)(nelx+1) points, 3 doubles each, laid out
 * [K][J][I][xyz]; element (ex,ey,ez) is the trilinear map of its 8 corners.
 * Periodic directions need flat, translation-equivalent boundary planes.
 * Computes on the device, in FP64: GLL nodes/weights, D, node coordinates,
 * J^{-1}, the six geometric factors G and the mass B (plus FP32 copies).
 * Errors: SEM_ERR_ARG, SEM_ERR_BAD_MESH (some |J| <= 0), SEM_ERR_NOMEM,
 * SEM_ERR_CUDA.  On success *out owns all library memory. */
SEM_API int sem_setup(int N, int nelx, int nely, int nelz, const double extents[3],
              const int periodic[3], const double *vertices, sem_ctx **out);

/* Free a context (NULL is allowed).  Synchronises the device first. */
SEM_API void sem_destroy(sem_ctx *ctx);

/* Sizes of a context. */
SEM_API int sem_get_info(const sem_ctx *ctx, sem_ctx_info *info);

/* Message for an error code (static string). */
SEM_API const char *sem_strerror(int code);

/* Text of the last CUDA runtime error seen by this host thread (for
 * SEM_ERR_CUDA); empty if none. */
SEM_API const char *sem_last_cuda_error(void);

/* Status of the bounded device-side waits of asynchronous stand-alone kernels
 * (the bulk-copy staged operator) since the previous call: SEM_OK, or
 * SEM_ERR_TIMEOUT if a staged copy did not arrive in time (its output is then
 * incomplete).  Synchronises the device; clears the status. */
SEM_API int sem_device_status(sem_ctx *ctx);

/* Node coordinates: xyz holds 3 E-vectors (x, then y, then z), FP64. */
SEM_API int sem_coords(sem_ctx *ctx, double *xyz, void *stream);

/* Geometric factors as computed by sem_setup: out holds 7 E-vectors, FP64, in
 * the order G11, G22, G33, G12, G13, G23, B, where
 *   B = w_i w_j w_k |J|,  G_ab = B sum_c (dr_a/dx_c)(dr_b/dx_c). */
SEM_API int sem_geom(sem_ctx *ctx, double *out, void *stream);

/* Local Helmholtz operator, ax_helm (Sec. 4, Table 2 rows B-6, B-7):
 *   w_e = h1 sum_{a,b} D_a^T G_ab D_b u_e + h2 B u_e   for every element e,
 * with D_r = I x I x D, D_s = I x D x I, D_t = D x I x I.  Not assembled
 * (follow with sem_dssum).  u and w must not overlap.  dtype selects the
 * arithmetic; SEM_BF16_TC / SEM_F16_TC round u and the intermediate fluxes
 * to 16 bits for tensor-core contractions with FP32 accumulation. */
SEM_API int sem_ax(sem_ctx *ctx, const void *u, void *w, double h1, double h2, sem_dtype dtype,
           void *stream);

/* Entries of sem_tune_ax's ms array. */
#define SEM_TUNE_MAX 16

/* Autotuner of sem_ax's kernel choice for the context's order N and dtype.
 * Times every candidate kernel and tile shape reps times on the context's
 * solver workspace (scratch between solves; no allocation), stores the
 * fastest for this process and returns it in *best; ms (NULL, or
 * SEM_TUNE_MAX entries) receives the average time of each candidate (-1
 * where a candidate does not apply).  Synchronous.  Candidates:
 *  - SEM_F32: 0 = direct loads, 1 = bulk-copy staged, 256 threads x 2 stages,
 *    2 = staged, 128 threads x 3 stages;
 *  - SEM_F64 with even N+1 <= 12: the float-pair folded kernel with
 *    0 = 256/(N+1)^2 elements per block and block-wide barriers, 1 = one
 *    hardware barrier per element where (N+1)^2 is a multiple of 32 (else as
 *    0), 2 = half the elements per block; the block-floating-point kernel
 *    with 3 = direct loads, 4 = direct loads and paired f32x2 instructions,
 *    5 = u staged by bulk copies, 6 = staged and paired, 7 = staged with half
 *    the elements per block, 8 = staged with one element per block,
 *    9 and 10 = as 8 with register budgets for 20 and 24 warps per SM
 *    (the staged forms fall back to 3 or 4 for u in host memory or not
 *    16-byte aligned);
 *  - SEM_F64_NATIVE with even N+1: 0 = the folded (even-odd) kernel,
 *    1 = the unfolded kernel;
 *  - other cases have one candidate, reported as 0 ms. */
SEM_API int sem_tune_ax(sem_ctx *ctx, sem_dtype dtype, int reps, double *ms, int *best);

/* Selects sem_ax's kernel for order N and dtype in this process (e.g. from a
 * cached tuning result); -1 restores the built-in per-order default, which
 * applies until a variant is set. */
SEM_API int sem_set_ax_variant(int N, sem_dtype dtype, int variant);

/* Direct-stiffness sum in place (Sec. 2, gather/scatter): every local copy of
 * a unique node receives the sum of all its copies (Q Q^T u).  Deterministic:
 * no atomics, a fixed summation order per unique node.  dtype SEM_F64 (double)
 * or SEM_F32 (float; the TC dtypes are treated as SEM_F32). */
SEM_API int sem_dssum(sem_ctx *ctx, void *u, sem_dtype dtype, void *stream);

/* Inverse assembled Jacobi diagonal, FP64 E-vector:
 *  minv = 1 / dssum( h1 [ sum_l D_li^2 G11(l,j,k) + sum_l D_lj^2 G22(i,l,k)
 *                        + sum_l D_lk^2 G33(i,j,l) + 2 D_ii D_jj G12
 *                        + 2 D_ii D_kk G13 + 2 D_jj D_kk G23 ] + h2 B ). */
SEM_API int sem_jacobi(sem_ctx *ctx, double h1, double h2, double *minv, void *stream);

/* Solver options.  tol: stopping tolerance on the assembled residual norm
 * ||r|| = sqrt(sum_local r^2 / mult); relative to ||b|| unless abs_tol != 0.
 * inner: the operator precision; SEM_F64 runs plain FP64 PCG, the other three
 * run FP64 iterative refinement around an inner PCG in that precision
 * (vectors FP32, dot products FP64) with relative tolerance inner_tol.
 * SEM_F64 with a relative tol below 1e-11 runs on the native FP64 operator
 * (SEM_F64_NATIVE): the FP64-accurate operators on the FP32 pipes carry a
 * relative error of a few 1e-13 per application, the size of such a residual,
 * and on a singular periodic Poisson problem their error on the constant
 * mode can end the solve in SEM_ERR_BREAKDOWN.
 * maxit bounds the PCG iterations (total inner iterations for refinement),
 * max_outer the refinement steps.  wait_timeout_s bounds every device-side
 * wait of the persistent solver (<= 0 selects 10 s); when one runs out the
 * solve ends with SEM_ERR_TIMEOUT and the context stays usable. */
typedef struct {
    double tol;
    int abs_tol;
    int maxit;
    sem_dtype inner;
    double inner_tol;
    int max_outer;
    double wait_timeout_s;
} sem_solve_opts;

/* Filled after the stream is synchronised. */
typedef struct {
    int status;         /* SEM_OK, SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN, SEM_ERR_TIMEOUT */
    int iters;          /* PCG iterations (sum of inner iterations under refinement) */
    int outer_iters;    /* refinement steps (0 for plain FP64 PCG) */
    double final_rnorm; /* FP64 assembled residual norm at exit */
    double bnorm;       /* FP64 assembled norm of the (mean-free when h2 == 0) RHS */
} sem_solve_info;

/* Default options: tol 1e-10 relative, maxit 20000, inner SEM_F64,
 * inner_tol 1e-4, max_outer 50, wait_timeout_s 0 (10 s). */
SEM_API void sem_solve_opts_default(sem_solve_opts *opts);

/* Jacobi-PCG on dssum(A) x = b with A = h1 D^T G D + h2 B (Sec. 1.1: CG with
 * the Jacobi preconditioner; Sec. 2: reductions in fp64).  b: assembled RHS
 * (continuous E-vector), FP64.  x: FP64 E-vector, initial guess on entry,
 * solution (or last iterate) on exit.  With h2 == 0 the constants span the
 * null space: b loses its mean before the iteration and x its B-weighted mean
 * after it.  The whole solve is one persistent cooperative kernel launch
 * (graph capturable); every wait inside it is bounded (SEM_ERR_TIMEOUT).
 * info: NULL for a fully asynchronous call (read it later with
 * sem_last_solve_info after synchronising), else the call synchronises the
 * stream, fills *info and returns info->status. */
SEM_API int sem_pcg_solve(sem_ctx *ctx, const double *b, double *x, double h1, double h2,
                  const sem_solve_opts *opts, sem_solve_info *info, void *stream);

/* Status of the last solve enqueued on ctx (valid after a stream sync). */
SEM_API int sem_last_solve_info(sem_ctx *ctx, sem_solve_info *info);

/* nprob independent solves in one persistent launch.  ctxs[p], b[p], x[p],
 * h1[p], h2[p] as in sem_pcg_solve (device pointers only); contexts may
 * differ in N and element count and may repeat.  infos (host, nprob entries)
 * may be NULL for an asynchronous call.  All problems use opts. */
SEM_API int sem_pcg_solve_batched(int nprob, sem_ctx *const *ctxs, const double *const *b,
                          double *const *x, const double *h1, const double *h2,
                          const sem_solve_opts *opts, sem_solve_info *infos, void *stream);

/* Largest problem (local nodes E (N+1)^3) that sem_pcg_solve_noalloc accepts. */
#define SEM_NOALLOC_MAX_NODES 1000000

/* FP64 Jacobi-PCG that allocates nothing -- an addition of this library; the
 * paper has no counterpart.  It is meant for callers that cannot call
 * cudaMalloc: code whose device memory is owned by another allocator (a
 * framework's caching allocator, a plugin host, a service with a fixed memory
 * plan), and code that must avoid cudaMalloc's implicit device
 * synchronisation.  It needs no context: the caller passes the mesh shape (N,
 * nelx, nely, nelz, periodic), the geometric factors geom as a device FP64
 * array laid out element by element, [E][7][(N+1)^3] with components G11 G22
 * G33 G12 G13 G23 B (the factors sem_geom exports, regrouped per element), the
 * assembled RHS b and the initial guess / solution x (device FP64 E-vectors),
 * and host opts/info (info is required; opts->inner must be SEM_F64 or
 * SEM_F64_NATIVE, and either runs the native-FP64 operator: the arithmetic of
 * sem_pcg_solve with inner = SEM_F64_NATIVE, same persistent kernel).  Every
 * scratch vector, partial sum and the solver state live in one file-scope
 * device array of fixed size (about 33 MB, held on every GPU that loads the
 * library until the process exits), so problems with more than
 * SEM_NOALLOC_MAX_NODES local nodes return SEM_ERR_TOO_LARGE.  The first call
 * on a device looks up that array's device address (once per device, cached
 * for the process; a cudaDeviceReset of that device makes the cached address
 * stale, so calls after a reset are not supported).  All calls share the one
 * array, which keeps the previous call's contents (the call clears the solver
 * state itself): calls that overlap on the GPU (from several streams or host
 * threads) race and give wrong results.  The call reads the mesh volume back
 * to the host, synchronises the stream before returning and returns
 * info->status. */
SEM_API int sem_pcg_solve_noalloc(int N, int nelx, int nely, int nelz, const int periodic[3],
                                  const double *geom, const double *b, double *x, double h1,
                                  double h2, const sem_solve_opts *opts, sem_solve_info *info,
                                  void *stream);

/* Autotuner of the inner path of refinement for the context's order N.  The
 * candidates are the two FP32-accurate inner operators: 0 = the FP32
 * CUDA-core operator (256/(N+1)^2 elements per 256-thread block, slabs in
 * shared memory per element) and 1 = the split-operand FP16 tensor-core
 * operator (SEM_F16X2_TC: one element per warp, 8 per block; N <= 7 only).
 * Each runs `iters` inner PCG iterations (a Helmholtz problem on the
 * context's mesh, one persistent launch) after one untimed run; ms (NULL or
 * 2 entries) receives the time per inner iteration (-1 where a candidate does
 * not apply) and *best the faster path, which becomes the order's choice for
 * solves with inner = SEM_F32_TUNED in this process (and in one batched launch
 * every problem takes its own order's path).  Allocates two E-vectors for the
 * run and frees them; synchronous. */
SEM_API int sem_tune_inner(sem_ctx *ctx, int iters, double *ms, int *best);

/* Sets the inner path of order N for SEM_F32_TUNED (e.g. from a cached tuning
 * result): 0 FP32 CUDA cores, 1 split FP16 tensor cores (N <= 7). */
SEM_API int sem_set_inner_path(int N, int path);

/* ---- Pressure solver: flexible GMRES + hybrid Schwarz multigrid (Sec. 1, Sec. 3) ---- */

typedef struct sem_hsmg sem_hsmg;

/* Hybrid Schwarz multigrid preconditioner of h1 A + h2 B on ctx's mesh (the
 * paper's pressure solver uses GMRES with a three-level HSMG whose coarse
 * problem is solved by CG + Jacobi).  nlev = 1..3 levels of polynomial orders
 * orders[0] = ctx's N > orders[1] > ... (e.g. {N, 3, 1}); N <= 9.  One
 * application is a V-cycle: on every level but the last, an overlapping
 * Schwarz smoother (element solves of the separable box operator extended to
 * the neighbours' first interior GLL nodes, by fast diagonalisation, averaged
 * over shared nodes), the level residual, restriction (transpose of Lagrange
 * interpolation); on the last level Jacobi-PCG in FP64 to relative tolerance
 * coarse_tol within coarse_maxit iterations; then prolongation and
 * correction.  dtype: SEM_F32 or SEM_F64, the precision of the V-cycle
 * (smoother, transfers, level operators).  Creates one context per coarser
 * level (sem_setup on the same vertices) and allocates about 3 E-vectors per
 * level plus the factor tables; the caller's ctx must outlive the object.
 * The coarse solve runs on workspace slot 0 of the coarsest level's context,
 * which is the caller's ctx when nlev = 1 (the slot sem_pcg_solve uses).  One
 * call at a time per object (its vectors are shared by its calls).
 * SEM_ERR_ARG: bad orders, N > 9, dtype, h1 <= 0, h2 < 0, coarse_tol <= 0 or
 * coarse_maxit < 1; SEM_ERR_NOMEM. */
SEM_API int sem_hsmg_create(sem_ctx *ctx, int nlev, const int *orders, double h1, double h2,
                            sem_dtype dtype, double coarse_tol, int coarse_maxit, sem_hsmg **out);

/* z = M^{-1} r: one V-cycle (r, z: FP64 E-vectors in device memory, continuous
 * across shared nodes as an assembled residual is; z is continuous).
 * Stream-ordered.  SEM_ERR_ARG: NULL or host pointers. */
SEM_API int sem_hsmg_apply(sem_hsmg *hsmg, const double *r, double *z, void *stream);

/* Flexible GMRES(restart) on dssum(h1 A + h2 B) x = b with the operator and
 * coefficients of hsmg's finest level, right-preconditioned by one V-cycle per
 * iteration (precond != 0) or not at all.  b, x: FP64 E-vectors in device
 * memory; x holds the initial guess and receives the solution.  opts: tol,
 * abs_tol and maxit as for sem_pcg_solve (inner, inner_tol, max_outer,
 * wait_timeout_s unused).  The operator is sem_ax's FP64-accurate one (the
 * native FP64 operator for a relative tol below 1e-11); inner products are
 * FP64 over unique nodes; with h2 == 0 b loses its mean and x its B-weighted
 * mean.  restart: 1..64 Krylov vectors per cycle (storage: 2 restart + 3
 * FP64 E-vectors, allocated on first use and kept).  Synchronises the stream
 * (the host solves the Hessenberg least-squares problem and reads three
 * inner-product sets per iteration).  Converged (SEM_OK) when the true
 * residual, computed at the end of every cycle, meets the target; below
 * 1e-8 ||b|| it is computed with the native FP64 operator (the FP64-accurate
 * operator's rounding floor, a few 1e-13 relative per application times
 * ||A|| ||x||, can reach that level), so that the cycles act as the inner
 * solves of an FP64 refinement.  A cycle that meets its own Arnoldi estimate
 * without halving the true residual ends the solve (SEM_ERR_NOT_CONVERGED).
 * info: iters (GMRES iterations), outer_iters (restarts), final_rnorm (true
 * residual), bnorm.  Returns info->status (SEM_OK, SEM_ERR_NOT_CONVERGED,
 * SEM_ERR_BREAKDOWN) or an error. */
SEM_API int sem_gmres_solve(sem_hsmg *hsmg, int precond, const double *b, double *x,
                            const sem_solve_opts *opts, int restart, sem_solve_info *info,
                            void *stream);

/* Free (NULL allowed; synchronises the device; destroys the coarser contexts). */
SEM_API void sem_hsmg_destroy(sem_hsmg *hsmg);

/* ---- Taylor-Green vortex stepper (Sec. 3) ---- */

typedef struct {
    double t, ke, enstrophy;   /* KE = 1/(2V) sum_local B |u|^2, enstrophy likewise with curl u */
    int iters[4];              /* pressure, u, v, w solver iterations */
    int status;
    double dt;                 /* size of the step */
    double cfl;                /* CFL number of the new velocity for that step: dt times the
                                  largest sum_a |U_a| / dxi_a over the local nodes, U_a =
                                  sum_c (dr_a/dx_c) u_c, dxi_a the GLL gap at the node's
                                  index along a (the smaller neighbouring gap) */
} sem_tgv_diag;

/* Stepper on a periodic context (Sec. 3: the P_N-P_N splitting with BDF3/EXT3
 * and 3/2-rule dealiasing; N <= 9).  nu: viscosity; dt: time step (fixed
 * until sem_tgv_set_dt changes it or turns on the CFL-controlled step).
 * op: precision of the dealiased convection: SEM_F64 (FP64-accurate, float
 * pairs on the FP32 pipes), SEM_F64_NATIVE (FP64 arithmetic) or SEM_F32
 * (histories, right-hand sides, refinement residuals and diagnostics stay FP64).  vel / pres: options
 * of the velocity Helmholtz and pressure Poisson solves (NULL = defaults: FP64
 * PCG; with op = SEM_F32 the default pressure solve is an FP32 inner PCG inside
 * FP64 refinement).  The solves' inner field selects their precision.
 * The stepper keeps a reference to ctx (which must outlive it) and solves on
 * the context's workspace slots 4-7; it allocates about 32 FP64 E-vectors plus
 * J^-1 and float-pair tables on the device (SEM_ERR_NOMEM if they do not fit).
 * SEM_ERR_ARG: NULL ctx or out, nu or dt not positive, an unsupported op, a
 * context that is not periodic in all three directions, or N > 9.  The state
 * is zero until sem_tgv_set. */
SEM_API int sem_tgv_init(sem_ctx *ctx, double nu, double dt, sem_dtype op, const sem_solve_opts *vel,
                 const sem_solve_opts *pres, sem_tgv **out);

/* Three-level precision policy of the stepper (Sec. 2, Fig. 2; the configurations
 * of Table 2).  One rule gives, per program block, the precision of each role:
 *  - sem: compute precision of the dealiased convection (the SEM block):
 *    SEM_F64 (FP64-accurate on the FP32 pipes), SEM_F64_NATIVE, SEM_F32, or the
 *    kernel-level overrides SEM_F16_TC / SEM_BF16_TC =
 *    every operand of its contractions rounded to FP16 / BF16, FP32 accumulation;
 *  - vel, pres: compute precision of the three velocity Helmholtz solves and of
 *    the pressure Poisson solve: SEM_F64 (PCG on the FP64-accurate operator),
 *    SEM_F64_NATIVE, SEM_F32 (FP32 inner PCG inside FP64 refinement to the same
 *    tolerance) or the kernel-level ax_helm overrides SEM_F16_TC / SEM_BF16_TC
 *    (16-bit tensor-core operator in that inner PCG);
 *  - storage: the global cap rp on stored state: SEM_F64, or SEM_F32 = the
 *    velocity and convection histories are held in FP32 buffers (18 FP32
 *    E-vectors, allocated by the first sem_tgv_set_policy whose rules ask for
 *    them; read and widened by the kernels that use them), and the pressure,
 *    which is the pressure solve's FP64 iterate, is rounded to FP32 values
 *    where it is stored.  A change of storage between two steps moves the
 *    histories to the other buffers (rounding to nearest towards FP32).
 * Accumulation (dot products, norms, refinement residuals, BDF/EXT sums, the
 * KE / enstrophy diagnostics) is FP64 under every rule.  first_step: the rule
 * applies from that step on (1-based; <= 1 = from the first step). */
typedef struct {
    int first_step;
    sem_dtype sem, vel, pres, storage;
} sem_tgv_policy;

#define SEM_TGV_MAX_RULES 8

/* Replace the stepper's policy schedule by n <= SEM_TGV_MAX_RULES rules in
 * non-decreasing first_step order.  At each step the last rule whose first_step
 * <= that step is in force; before the first rule starts (and with n = 0) the
 * precisions given to sem_tgv_init apply.  A change of rule between two steps
 * re-captures the step graph.  Returns SEM_ERR_ARG for an unsupported
 * precision or an unsorted schedule, SEM_ERR_NOMEM if the FP32 history
 * buffers do not fit (the previous schedule then stays). */
SEM_API int sem_tgv_set_policy(sem_tgv *tgv, int n, const sem_tgv_policy *rules);

/* Projection of the pressure solve onto previous solutions (Sec. 3: the
 * pressure solver keeps a projection space of dimension 20; the A-conjugate
 * projection of Fischer, CMAME 163, 1998).  max_vectors in 1..32 keeps an
 * A-orthonormal basis of up to that many earlier pressure solutions: each
 * pressure solve starts from the A-projection of its right-hand side onto the
 * basis and iterates only on the remainder, whose solution (A-orthogonalised
 * twice) joins the basis; a full basis restarts from the latest solution.
 * 0 turns it off (the default).  Allocates 2 max_vectors + 5 FP64 E-vectors on
 * the context's device (SEM_ERR_NOMEM if they do not fit); synchronises the
 * device; the next step re-captures the step graph.  The basis starts empty. */
SEM_API int sem_tgv_set_projection(sem_tgv *tgv, int max_vectors);

/* Step size control (Sec. 3: the step adapts to hold CFL = 0.4).  dt > 0 sets
 * the size of the next step (0 keeps it).  cfl_target > 0 turns on the
 * CFL-controlled step: after each step the host reads that step's CFL number
 * (see sem_tgv_diag) and takes the next step dt * f, f = cfl_target / CFL
 * clamped to [0.5, 1.1], capped by dt_max when dt_max > 0 (a zero CFL keeps the
 * step); cfl_target = 0 keeps the step fixed.  Unequal steps take the
 * variable-step BDF3/EXT3 coefficients of the last three step sizes; the
 * history levels set by sem_tgv_set count as steps of the current size.  A
 * CFL-controlled run synchronises the stream once per step and launches every
 * step directly (no graph replay); a changed fixed step re-captures the step
 * graph once three steps of the new size have run.  SEM_ERR_ARG: NULL tgv or
 * a negative or NaN argument. */
SEM_API int sem_tgv_set_dt(sem_tgv *tgv, double dt, double cfl_target, double dt_max);

/* Pressure solver of the stepper: kind 0 = Jacobi-PCG in the persistent
 * kernel (the default), 1 = flexible GMRES(restart) preconditioned by the
 * hybrid Schwarz multigrid (Sec. 1, Sec. 3: GMRES + three-level HSMG with a
 * CG + Jacobi coarse solve): levels N, 3, 1 (N, 2, 1 for N = 3, 4; N, 1 for
 * N = 2), V-cycle in vcycle precision (SEM_F32 or SEM_F64), coarse PCG to
 * relative tolerance 0.1.  The pressure options' tol, abs_tol and maxit
 * apply; their inner field does not (the V-cycle precision is vcycle).  With
 * kind 1 every step launches directly (GMRES reads inner products back to the
 * host), the projection (sem_tgv_set_projection) still applies, and the
 * pressure entry of sem_tgv_diag counts GMRES iterations.  Synchronises the
 * device; allocates the hierarchy (about 3 E-vectors per level, the coarser
 * levels' contexts) and, on the first solve, 2 restart + 3 FP64 E-vectors.
 * SEM_ERR_ARG: NULL tgv, kind outside 0..1, restart outside 1..64 or an
 * unsupported vcycle; SEM_ERR_NOMEM. */
SEM_API int sem_tgv_set_pressure_solver(sem_tgv *tgv, int kind, int restart, sem_dtype vcycle);

/* Set the state at history level (0 = u^n, 1 = u^{n-1}, 2 = u^{n-2}) from
 * FP64 E-vectors u, v, w (and p for level 0; may be NULL), each device or host
 * memory (copied); step is the number of steps already taken (selects the
 * startup order: 0 = first order next), t the time.  Levels 1 and 2 also
 * evaluate that level's convective term.  Synchronises the stream.
 * SEM_ERR_ARG: NULL tgv, u, v or w, level outside 0..2, or step < 0. */
SEM_API int sem_tgv_set(sem_tgv *tgv, int level, const double *u, const double *v, const double *w,
                const double *p, int step, double t, void *stream);

/* Advance nsteps P_N-P_N steps (BDF3/EXT3, 3/2-rule dealiasing).  diag: host
 * array of nsteps entries or NULL; when given, the call synchronises (after
 * every 4096 steps at most: the device keeps a ring of 4096 log entries) and
 * returns the first nonzero solve status of those steps
 * (SEM_ERR_NOT_CONVERGED, SEM_ERR_BREAKDOWN or SEM_ERR_TIMEOUT; the steps still
 * ran, with the last iterate of that solve); without diag the call is
 * stream-ordered and returns SEM_OK or a launch error (a CFL-controlled run
 * synchronises once per step).  With a fixed step, from the third step of one
 * size on each step is one CUDA graph replay (captured on the second such step
 * after setup or any policy, projection or step-size change; direct launches
 * if the capture fails) when stream is not NULL.
 * SEM_ERR_ARG: NULL tgv or nsteps < 0. */
SEM_API int sem_tgv_step(sem_tgv *tgv, int nsteps, sem_tgv_diag *diag, void *stream);

/* Copy out u^n, v^n, w^n, p^n (FP64 E-vectors, device or host memory; any
 * may be NULL); stream-ordered (a host destination is valid after a stream
 * synchronisation).  SEM_ERR_ARG: NULL tgv. */
SEM_API int sem_tgv_get(sem_tgv *tgv, double *u, double *v, double *w, double *p, void *stream);

/* Kinetic energy and enstrophy of the current state (Sec. 4.2 diagnostics;
 * host doubles, FP64-accurate reductions); synchronises the stream.  SEM_ERR_ARG: a
 * NULL argument. */
SEM_API int sem_tgv_energy(sem_tgv *tgv, double *ke, double *enstrophy, void *stream);

/* Free a stepper (NULL is allowed); synchronises the device first.  The
 * context stays valid. */
SEM_API void sem_tgv_destroy(sem_tgv *tgv);

#ifdef __cplusplus
}
#endif
#endif /* SEM_H */
