// solver.cuh -- persistent, cooperative Jacobi-PCG / FP64 iterative refinement.
//
// One launch runs a whole solve (or a batch of independent solves).  Every
// problem carries a small state machine; all problems advance together in
// "grid steps".  In a step each problem executes the work items of its
// current phase (element groups, chunks of unique nodes or chunks of local
// nodes), every CTA adds its FP64 partial sums, and a reducing grid barrier
// ends the step: the last CTA to arrive sums the partials of every problem in
// a fixed order (deterministic), advances each state machine, publishes the
// next schedule and releases the others.  Every wait is bounded in time; a
// CTA that gives up raises SEM_ERR_TIMEOUT and the whole grid exits.
//
// Phases of one problem (Sec. 1.1: CG with Jacobi; Sec. 2: dot products and
// norms reduced in fp64):
//   JAC    local   minv = local diagonal of A
//   JACGS  unique  minv = 1/dssum(minv);  sum b  (mean removal when h2 == 0)
//   AX0    element w = A x                                      (FP64)
//   R0     unique  r = b' - dssum(w); <r,r>, <r,z>, <b',b'>      (plain PCG)
//   A      element x += alpha p (previous step); p = z + beta p; w = A p; <p,w>
//   C      unique  r -= alpha dssum(w); <r,r>, <r,z>
//   XUPD   local   x += alpha p (the last step, after convergence)
//   R64    unique  r = b' - dssum(w); <r,r>, <b',b'>            (refinement)
//   INIT32 unique  r32 = r / ||r||; d = 0; <r32,r32>, <r32,z32>
//   A32    element d += alpha p32; p32 = z32 + beta p32; w32 = A32 p32; <p32,w32>
//   C32    unique  r32 -= alpha dssum(w32); <r32,r32>, <r32,z32>
//   UPD    local   p = x (kept until the next FP64 residual accepts the step);
//                  x += ||r|| (d + alpha p32 when that last step is pending)
//   XREST  local   x = p: a refinement step that raised the FP64 residual is
//                  undone, so a solve never returns an iterate worse than the
//                  one it had before that step
//   FINAL  local   sum B x              (h2 == 0: remove the B-weighted mean)
//   SHIFT  local   x -= sum(B x) / sum(B)
// The inner product <a,b> = sum_local a b / mult is evaluated over unique
// nodes, where it is a plain sum; <p, dssum(Ap)> equals sum_local p (Ap)
// for a continuous p, which lets the element phase produce it directly.
// Unique-node items are a chunk of 256 consecutive gx on SEM_UQ_ROWS rows
// (gy, gz): the y/z copies are computed once per row, the x copies once per
// thread, and all loads of a thread are issued before any store.
#pragma once

#include <type_traits>

#include "ax.cuh"
#include "ax_bfp.cuh"
#include "ax_df.cuh"
#include "ax_dfeo.cuh"
#include "ax_tc.cuh"
#include "common.cuh"
#include "gs.cuh"
#include "tma.cuh"

#define SEM_MAXP 64
#define SEM_SOLVE_THREADS 256
#define SEM_UQ_ROWS 4
#ifndef SEM_SOLVE_F64_MINB
#define SEM_SOLVE_F64_MINB 2
#endif
#ifndef SEM_SOLVE_F32_MINB
#define SEM_SOLVE_F32_MINB 3
#endif
// Element phases prefetch their group's geometric factors into L2.
#ifndef SEM_SOLVE_GEO_PREFETCH
#define SEM_SOLVE_GEO_PREFETCH 1
#endif
// FP64-accurate element phases of even orders use the folded operator.
#ifndef SEM_SOLVE_DF_FOLDED
#define SEM_SOLVE_DF_FOLDED 1
#endif
// ... and, for even N+1 <= 12, the block-floating-point operator.
#ifndef SEM_SOLVE_BFP
#define SEM_SOLVE_BFP 1
#endif

// Which element operators a solver kernel carries (keeps each kernel's
// register budget to what its mode needs).
// MODE_F64 evaluates the FP64 operator on the FP32 pipes (float pairs,
// ax_df.cuh); MODE_F64N uses native FP64 arithmetic.
enum SolveMode { MODE_F64 = 0, MODE_F32 = 1, MODE_TC = 2, MODE_F64N = 3 };

enum SolvePhase {
    PH_JAC = 0, PH_JACGS, PH_AX0, PH_R0, PH_A, PH_C, PH_R64, PH_INIT32, PH_A32, PH_C32, PH_UPD,
    PH_FINAL, PH_SHIFT, PH_XUPD, PH_XREST, PH_DONE
};

struct ProbDesc {
    int n, NE, NE32, singular;  // NE: elements per group (CUDA cores); NE32: inner operator
    int tc;                     // inner path of a MODE_TC launch: 0 FP32 CUDA cores, 1 BF16, 2 FP16,
                                // 3 FP16 x2, 4 BF16 x3 tensor cores
    int jac_cached;             // minv (and minv32 if mixed) already hold this problem's Jacobi inverse
    int64_t E, nL, nG;
    GsDesc gs;
    double volume, h1, h2;
    const double *geo64;
    const float *geo32;
    const dfp *geodf;
    const double *D64;
    const float *D32;
    const dfp *Ddf;
    const dfp *Ddfeo;   // folded half tables (even orders)
    const double *b;
    double *x;
    double *r, *p, *w, *minv;
    float *r32, *p32, *w32, *d32, *minv32;
};

struct PState {
    int phase, iters, outer, inner_iters, status, first, nvals, pending;
    double rz, alpha, beta, bnorm, rnorm, target, bmean, scale, prev_rnorm, inner_target, shift;
};

struct SyncState {
    unsigned count, gen;
    int err, finished;
};

template <int MAXP>
struct SolveParams {
    int nprob, mixed, inner_tc, abs_tol, maxit, max_outer;
    double tol, inner_tol;
    long long timeout_ns;
    SyncState *sync;
    PState *st;
    double *partials;   // [gridDim][MAXP][3]
    int *sched;         // phase[MAXP], then offsets[MAXP + 1]
    ProbDesc prob[MAXP];
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long sem_globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int phase_nvals(int ph)
{
    switch (ph) {
        case PH_JACGS: return 1;
        case PH_R0: return 3;
        case PH_A: case PH_A32: return 1;
        case PH_C: case PH_C32: case PH_R64: case PH_INIT32: return 2;
        case PH_FINAL: return 1;
        default: return 0;
    }
}

__device__ __forceinline__ int64_t phase_items(const ProbDesc &P, int ph)
{
    switch (ph) {
        case PH_JAC: case PH_UPD: case PH_FINAL: case PH_SHIFT: case PH_XUPD: case PH_XREST:
            return (P.nL + SEM_SOLVE_THREADS - 1) / SEM_SOLVE_THREADS;
        case PH_JACGS: case PH_R0: case PH_C: case PH_R64: case PH_INIT32: case PH_C32: {
            const int64_t nxch = (P.gs.ngx + SEM_SOLVE_THREADS - 1) / SEM_SOLVE_THREADS;
            const int64_t rows = (int64_t)P.gs.ngy * P.gs.ngz;
            return nxch * ((rows + SEM_UQ_ROWS - 1) / SEM_UQ_ROWS);
        }
        case PH_AX0: case PH_A:
            return (P.E + P.NE - 1) / P.NE;
        case PH_A32:
            return (P.E + P.NE32 - 1) / P.NE32;
        default:
            return 0;
    }
}

// FP32 dot products accumulated on the FP32 pipes: every product exact
// (TwoProd), every sum error-free (TwoSum), the errors gathered in A.e -- the
// compensated dot product of Ogita, Rump & Oishi, as accurate as summing the
// exact products in twice FP32 precision.  GB300 runs FP64 at 1/58 of the
// FP32 rate, so the per-node FP64 multiply-add (and two conversions) this
// replaces cost more issue time than the ten FP32 operations here.
__device__ __forceinline__ void dot2_acc(dfacc &A, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float ep = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(A.s, p);
    const float bv = __fsub_rn(s, A.s);
    const float t = __fadd_rn(__fsub_rn(A.s, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    A.s = s;
    A.e = __fadd_rn(A.e, __fadd_rn(t, ep));
}

__device__ __forceinline__ double dfacc_value(dfacc A) { return (double)A.s + (double)A.e; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds the block sum of v[0..2] into dst[0..2] (thread 0); all threads call.
__device__ __forceinline__ void block_accumulate(double v[3], double *s_red, double *dst)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) s_red[warp * 3 + k] = s;
        v[k] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int w = 0; w < SEM_SOLVE_THREADS / 32; ++w) s += s_red[w * 3 + k];
            dst[k] += s;
        }
    }
    __syncthreads();
}

// Thread 0 asks L2 for the geometric factors of the element group this block
// is about to work on (bytes [e0, e1) elements of a [E][7][NP^3] array of
// `wb`-byte words): the operator reads them after its gradient stage, about
// half an element phase later.  (A whole group ahead let L2 evict the element
// phase's output before the gather read it.)
template <int NP>
__device__ __forceinline__ void geo_prefetch(const void *geo, int64_t e0, int ne, int64_t E, int wb)
{
    constexpr int64_t N3 = NP * NP * NP;
    if (!SEM_SOLVE_GEO_PREFETCH || threadIdx.x != 0 || e0 >= E) return;
    const int64_t e1 = e0 + ne < E ? e0 + ne : E;
    l2_prefetch_span(geo, e0 * 7 * N3 * wb, e1 * 7 * N3 * wb);
}

// ---------------------------------------------------------------------------
// element items
// ---------------------------------------------------------------------------

// kind 0: w64 = A64 x;  kind 1: FP64 p-update + w = A p + <p,w>;
// kind 2: FP32 p32-update + w32 = A32 p32 + <p32,w32>.
template <int NP, int KIND>
__device__ __forceinline__ void elem_item(const ProbDesc &P, double alpha, double beta, int first,
                                          int64_t g, unsigned char *smem, double &acc)
{
    using C = AxCfg<NP>;
    using T = typename std::conditional<KIND == 2, float, double>::type;
    T *sm = reinterpret_cast<T *>(smem);
    T *sD = sm, *sDT = sm + NP * NP;
    const int grp = threadIdx.x / C::NP2;
    const int tid = threadIdx.x - grp * C::NP2;
    const bool inrange = grp < C::NE;
    const int64_t e = g * C::NE + grp;
    const bool active = inrange && e < P.E;
    T *su = sm + 2 * NP * NP + (size_t)(inrange ? grp : 0) * 3 * C::NP3;
    T *svr = su + C::NP3, *svs = svr + C::NP3;
    const int64_t off = (active ? e : 0) * C::NP3;
    const T *D = KIND == 2 ? (const T *)P.D32 : (const T *)P.D64;
    const T *geo = (KIND == 2 ? (const T *)P.geo32 : (const T *)P.geo64) + (active ? e : 0) * 7 * C::NP3;
    if (KIND == 2) geo_prefetch<NP>(P.geo32, g * C::NE, C::NE, P.E, 4);  // (native FP64: no gain)
    ax_load_D<NP, T>(D, sD, sDT);
    if (KIND == 0) {
        const double *x = P.x + off;
        double *w = P.w + off;
        auto load = [&](int q) { return (T)__ldcg(x + q); };
        auto store = [&](int q, T v, T) { w[q] = v; };
        ax_element<NP, T>(load, store, geo, (T)P.h1, (T)P.h2, sD, sDT, su, svr, svs, tid, active);
    } else if (KIND == 1) {
        const double *r = P.r + off, *mi = P.minv + off;
        double *p = P.p + off, *w = P.w + off, *x = P.x + off;
        auto load = [&](int q) {
            double pn = __ldcg(mi + q) * __ldcg(r + q);
            if (!first) {
                const double po = __ldcg(p + q);
                x[q] = fma(alpha, po, __ldcg(x + q));
                pn = fma(beta, po, pn);
            }
            p[q] = pn;
            return (T)pn;
        };
        auto store = [&](int q, T v, T u) {
            w[q] = v;
            acc = fma((double)u, (double)v, acc);
        };
        ax_element<NP, T>(load, store, geo, (T)P.h1, (T)P.h2, sD, sDT, su, svr, svs, tid, active);
    } else {
        const float *r = P.r32 + off, *mi = P.minv32 + off;
        float *p = P.p32 + off, *w = P.w32 + off, *d = P.d32 + off;
        const float b32 = (float)beta, a32 = (float)alpha;
        auto load = [&](int q) {
            float pn = __ldcg(mi + q) * __ldcg(r + q);
            if (!first) {
                const float po = __ldcg(p + q);
                d[q] = fmaf(a32, po, __ldcg(d + q));
                pn = fmaf(b32, po, pn);
            }
            p[q] = pn;
            return (T)pn;
        };
        dfacc dot = {0.f, 0.f};
        auto store = [&](int q, T v, T u) {
            w[q] = v;
            dot2_acc(dot, u, v);
        };
        ax_element<NP, T>(load, store, geo, (T)P.h1, (T)P.h2, sD, sDT, su, svr, svs, tid, active);
        acc += dfacc_value(dot);
    }
}

// FP64-accurate element phases on the FP32 pipes (float pairs):
// kind 0: w = A x;  kind 1: x += alpha p, p = z + beta p, w = A p, <p,w>.
template <int NP, int KIND>
__device__ __forceinline__ void elem_item_df(const ProbDesc &P, double alpha, double beta, int first,
                                             int64_t g, unsigned char *smem, double &acc)
{
    using C = AxDfCfg<NP>;
    dfp *sm = reinterpret_cast<dfp *>(smem);
    dfp *sD = sm, *sDT = sm + NP * NP;
    int *sexp = reinterpret_cast<int *>(sm + 2 * NP * NP + (size_t)C::NE * 3 * C::NP3);
    const int grp = threadIdx.x / C::NP2;
    const int tid = threadIdx.x - grp * C::NP2;
    const bool inrange = grp < C::NE;
    const int64_t e = g * C::NE + grp;
    const bool active = inrange && e < P.E;
    dfp *su = sm + 2 * NP * NP + (size_t)(inrange ? grp : 0) * 3 * C::NP3;
    dfp *svr = su + C::NP3, *svs = svr + C::NP3;
    const int64_t off = (active ? e : 0) * C::NP3;
    const dfp *geo = P.geodf + (active ? e : 0) * 7 * C::NP3;
    const float h1h = (float)P.h1, h2h = (float)P.h2;
    const dfp H1 = {h1h, (float)(P.h1 - (double)h1h)}, H2 = {h2h, (float)(P.h2 - (double)h2h)};
    geo_prefetch<NP>(P.geodf, g * C::NE, C::NE, P.E, 8);
    ax_df_load_D<NP>(P.Ddf, sD, sDT);
    int *myexp = sexp + (inrange ? grp : 0);
    if (KIND == 0) {
        const double *x = P.x + off;
        double *w = P.w + off;
        auto load = [&](int q) { return __ldcg(x + q); };
        auto store = [&](int q, double v) { w[q] = v; };
        ax_df_element<NP>(load, store, geo, H1, H2, sD, sDT, su, svr, svs, myexp, tid, active);
    } else {
        const double *r = P.r + off, *mi = P.minv + off;
        double *p = P.p + off, *w = P.w + off, *x = P.x + off;
        auto load = [&](int q) {
            double pn = __ldcg(mi + q) * __ldcg(r + q);
            if (!first) {
                const double po = __ldcg(p + q);
                x[q] = fma(alpha, po, __ldcg(x + q));
                pn = fma(beta, po, pn);
            }
            p[q] = pn;
            return pn;
        };
        auto store = [&](int q, double v) {
            w[q] = v;
            acc = fma(__ldcg(p + q), v, acc);
        };
        ax_df_element<NP>(load, store, geo, H1, H2, sD, sDT, su, svr, svs, myexp, tid, active);
    }
}

// The same phases with the folded (even-odd) float-pair operator, even orders.
template <int NP>
constexpr bool df_folded()
{
    // (and only while two blocks still fit on an SM)
    return SEM_SOLVE_DF_FOLDED && AxEoCfg<NP>::OK && AxEoCfg<NP>::THREADS <= SEM_SOLVE_THREADS &&
           ax_dfeo_smem_bytes<NP>() <= 112 * 1024;
}

template <int NP, int KIND>
__device__ __forceinline__ void elem_item_dfeo(const ProbDesc &P, double alpha, double beta, int first,
                                               int64_t g, unsigned char *smem, double &acc)
{
    using C = AxEoCfg<NP>;
    constexpr int HH = (NP / 2) * (NP / 2);
    dfp *sm = reinterpret_cast<dfp *>(smem);
    dfp *stab = sm;
    int *sexp = reinterpret_cast<int *>(sm + 4 * HH + (size_t)C::NE * 5 * C::SLAB);
    const int grp = threadIdx.x / C::NP2;
    const int tid = threadIdx.x - grp * C::NP2;
    const bool inrange = grp < C::NE;
    const int64_t e = g * C::NE + grp;
    const bool active = inrange && e < P.E;
    dfp *slab = sm + 4 * HH + (size_t)(inrange ? grp : 0) * 5 * C::SLAB;
    const int64_t off = (active ? e : 0) * C::NP3;
    const dfp *geo = P.geodf + (active ? e : 0) * 7 * C::NP3;
    const float h1h = (float)P.h1, h2h = (float)P.h2;
    const dfp H1 = {h1h, (float)(P.h1 - (double)h1h)}, H2 = {h2h, (float)(P.h2 - (double)h2h)};
    geo_prefetch<NP>(P.geodf, g * C::NE, C::NE, P.E, 8);
    for (int t = threadIdx.x; t < 4 * HH; t += blockDim.x) stab[t] = P.Ddfeo[t];
    int *myexp = sexp + (inrange ? grp : 0);
    if (KIND == 0) {
        const double *x = P.x + off;
        double *w = P.w + off;
        auto load = [&](int q) { return __ldcg(x + q); };
        auto store = [&](int q, double v) { w[q] = v; };
        ax_dfeo_element<NP>(load, store, geo, H1, H2, stab, slab, myexp, tid, active);
    } else {
        const double *r = P.r + off, *mi = P.minv + off;
        double *p = P.p + off, *w = P.w + off, *x = P.x + off;
        auto load = [&](int q) {
            double pn = __ldcg(mi + q) * __ldcg(r + q);
            if (!first) {
                const double po = __ldcg(p + q);
                x[q] = fma(alpha, po, __ldcg(x + q));
                pn = fma(beta, po, pn);
            }
            p[q] = pn;
            return pn;
        };
        auto store = [&](int q, double v) {
            w[q] = v;
            acc = fma(__ldcg(p + q), v, acc);
        };
        ax_dfeo_element<NP>(load, store, geo, H1, H2, stab, slab, myexp, tid, active);
    }
}

// The block-floating-point operator's tables for each even order, one copy
// per translation unit (constant-bank operands in the unrolled contractions);
// filled at context setup, outside any stream capture, by
// solver_upload_bfp_tables.
static __constant__ BfpTabs c_bfp_tabs[SEM_NPMAX / 2 + 1];

static inline int solver_upload_bfp_tables(int np, const void *tabs)
{
    if (np < 2 || np > SEM_NPMAX || np % 2 || !tabs) return SEM_ERR_ARG;
    SEM_CUDA(cudaMemcpyToSymbol(c_bfp_tabs, tabs, sizeof(BfpTabs), (size_t)(np / 2) * sizeof(BfpTabs)));
    return SEM_OK;
}

// Dynamic shared memory of a block-floating-point element phase: 2 KB of
// reduction words (zeroed at kernel start; each element leaves them zero),
// then the slabs.
#define SEM_BFP_RED_BYTES 2048

template <int NP>
constexpr bool solve_bfp()
{
    return SEM_SOLVE_BFP && BfpCfg<NP>::OK && NP <= 12 && BfpCfg<NP>::THREADS <= SEM_SOLVE_THREADS &&
           ax_bfp_smem_bytes_ne<NP, BfpCfg<NP>::NE>() + SEM_BFP_RED_BYTES <= 112 * 1024;
}


// FP64-accurate element phases with the block-floating-point operator:
// kind 0: w = A x;  kind 1: x += alpha p, p = z + beta p, w = A p, <p,w>.
template <int NP, int KIND>
__device__ __forceinline__ void elem_item_bfp(const ProbDesc &P, double alpha, double beta, int first,
                                              int64_t g, unsigned char *smem, double &acc)
{
    using C = BfpCfg<NP>;
    static_assert(8 * C::NE * sizeof(unsigned) <= SEM_BFP_RED_BYTES, "reduction words");
    unsigned *red = reinterpret_cast<unsigned *>(smem);
    dfp *slabs = reinterpret_cast<dfp *>(smem + SEM_BFP_RED_BYTES);
    const int grp = threadIdx.x / C::NP2;
    const bool inrange = grp < C::NE;
    // threads beyond the last whole element take part in the barriers only
    const int tid = inrange ? (int)threadIdx.x - grp * C::NP2 : -1;
    const int gs = inrange ? grp : 0;
    const int64_t e = g * C::NE + grp;
    const bool active = inrange && e < P.E;
    const int64_t off = (active ? e : 0) * C::NP3;
    const dfp *geo = P.geodf + (active ? e : 0) * 7 * C::NP3;
    const float h1h = (float)P.h1, h2h = (float)P.h2;
    const dfp H1 = {h1h, (float)(P.h1 - (double)h1h)}, H2 = {h2h, (float)(P.h2 - (double)h2h)};
    geo_prefetch<NP>(P.geodf, g * C::NE, C::NE, P.E, 8);
    const BfpTabs &T = c_bfp_tabs[NP / 2];
    dfp *slab = slabs + (size_t)gs * 3 * C::SLAB;
    if (KIND == 0) {
        const double *x = P.x + off;
        double *w = P.w + off;
        auto load = [&](int q) { return __ldcg(x + q); };
        auto store = [&](int q, double v) { w[q] = v; };
        ax_bfp_element<NP, false>(load, store, geo, H1, H2, T, slab, red + gs * 8, tid, active, [] {});
    } else {
        const double *r = P.r + off, *mi = P.minv + off;
        double *p = P.p + off, *w = P.w + off, *x = P.x + off;
        auto load = [&](int q) {
            double pn = __ldcg(mi + q) * __ldcg(r + q);
            if (!first) {
                const double po = __ldcg(p + q);
                x[q] = fma(alpha, po, __ldcg(x + q));
                pn = fma(beta, po, pn);
            }
            p[q] = pn;
            return pn;
        };
        auto store = [&](int q, double v) {
            w[q] = v;
            acc = fma(__ldcg(p + q), v, acc);
        };
        ax_bfp_element<NP, false>(load, store, geo, H1, H2, T, slab, red + gs * 8, tid, active, [] {});
    }
}

// FP64-accurate w = A x with the low-register float-pair operator (mixed
// modes: the FP64 residual of each refinement step); the NE elements of
// group g one after another.
template <int NP>
__device__ __forceinline__ void elem_item_lowreg(const ProbDesc &P, int64_t g, unsigned char *smem)
{
    constexpr int NP3 = NP * NP * NP;
    const float h1h = (float)P.h1, h2h = (float)P.h2;
    const dfp H1 = {h1h, (float)(P.h1 - (double)h1h)}, H2 = {h2h, (float)(P.h2 - (double)h2h)};
    for (int t = 0; t < P.NE; ++t) {
        const int64_t e = g * P.NE + t;
        if (e >= P.E) break;  // uniform across the block
        const double *x = P.x + e * NP3;
        double *w = P.w + e * NP3;
        auto load = [&](int q) { return __ldcg(x + q); };
        auto store = [&](int q, double v) { w[q] = v; };
        ax_df_element_lowreg<NP>(load, store, P.geodf + e * 7 * NP3, H1, H2, P.Ddf, smem);
    }
}

// TC inner operator (16-bit tensor-core contractions, FP32 vectors).  tc: 1
// BF16, 2 FP16 (plain rounding); 3 FP16 x2, 4 BF16 x3 (split operands, N+1 <= 8).
template <int NP>
__device__ __forceinline__ void elem_item_tc(const ProbDesc &P, double alpha, double beta, int first,
                                             int64_t g, int tc, unsigned char *smem, double &acc)
{
    const float b32 = (float)beta, a32 = (float)alpha;
    auto load = [&](int64_t q) {
        float pn = __ldcg(P.minv32 + q) * __ldcg(P.r32 + q);
        if (!first) {
            const float po = __ldcg(P.p32 + q);
            P.d32[q] = fmaf(a32, po, __ldcg(P.d32 + q));
            pn = fmaf(b32, po, pn);
        }
        P.p32[q] = pn;
        return pn;
    };
    dfacc dot = {0.f, 0.f};
    auto store = [&](int64_t q, float v, float u) {
        P.w32[q] = v;
        dot2_acc(dot, u, v);
    };
    if (tc == 3)
        ax_tc_split_group<NP, true>(load, store, P.geo32, P.D32, (float)P.h1, (float)P.h2, P.E, g, smem);
    else if (tc == 4)
        ax_tc_split_group<NP, false>(load, store, P.geo32, P.D32, (float)P.h1, (float)P.h2, P.E, g, smem);
    else
        ax_tc_group<NP>(load, store, P.geo32, P.D32, (float)P.h1, (float)P.h2, P.E, g, tc == 2, smem);
    acc += dfacc_value(dot);
}

template <int NP, int MODE>
__device__ __forceinline__ void elem_dispatch_np(const ProbDesc &P, int ph, double alpha, double beta,
                                                 int first, int64_t g, int tc, unsigned char *smem,
                                                 double &acc)
{
    if constexpr (MODE == MODE_F64 && solve_bfp<NP>()) {
        if (ph == PH_AX0)
            elem_item_bfp<NP, 0>(P, alpha, beta, first, g, smem, acc);
        else
            elem_item_bfp<NP, 1>(P, alpha, beta, first, g, smem, acc);
    } else if constexpr (MODE == MODE_F64 && df_folded<NP>()) {
        if (ph == PH_AX0)
            elem_item_dfeo<NP, 0>(P, alpha, beta, first, g, smem, acc);
        else
            elem_item_dfeo<NP, 1>(P, alpha, beta, first, g, smem, acc);
    } else if constexpr (MODE == MODE_F64) {
        if (ph == PH_AX0)
            elem_item_df<NP, 0>(P, alpha, beta, first, g, smem, acc);
        else
            elem_item_df<NP, 1>(P, alpha, beta, first, g, smem, acc);
    } else if constexpr (MODE == MODE_F64N) {
        if (ph == PH_AX0)
            elem_item<NP, 0>(P, alpha, beta, first, g, smem, acc);
        else
            elem_item<NP, 1>(P, alpha, beta, first, g, smem, acc);
    } else {
        if (ph == PH_AX0) {
            elem_item_lowreg<NP>(P, g, smem);
        } else if constexpr (MODE == MODE_TC) {
            // each problem of the launch has its own inner path
            if (P.tc == 0)
                elem_item<NP, 2>(P, alpha, beta, first, g, smem, acc);
            else
                elem_item_tc<NP>(P, alpha, beta, first, g, P.tc, smem, acc);
        } else
            elem_item<NP, 2>(P, alpha, beta, first, g, smem, acc);
    }
}

template <int MODE, int... NPs>
struct ElemDispatch;

template <int MODE>
struct ElemDispatch<MODE> {
    __device__ static void run(const ProbDesc &, int, double, double, int, int64_t, int,
                               unsigned char *, double &) {}
};

template <int MODE, int NP0, int... NPs>
struct ElemDispatch<MODE, NP0, NPs...> {
    __device__ static void run(const ProbDesc &P, int ph, double alpha, double beta, int first,
                               int64_t g, int tc, unsigned char *smem, double &acc)
    {
        if (P.n == NP0)
            elem_dispatch_np<NP0, MODE>(P, ph, alpha, beta, first, g, tc, smem, acc);
        else
            ElemDispatch<MODE, NPs...>::run(P, ph, alpha, beta, first, g, tc, smem, acc);
    }
};

// ---------------------------------------------------------------------------
// unique-node and local-node items (one node per thread)
// ---------------------------------------------------------------------------

// y/z copies of one row (gy, gz) of unique nodes: local offsets without the x part.
struct RowCopies {
    int m;
    int64_t off[4];
};

__device__ __forceinline__ void row_copies(const GsDesc &d, int row, RowCopies &R)
{
    const int gy = row % d.ngy, gz = row / d.ngy;
    int ey[2], iy[2], ez[2], iz[2];
    const int my = gs_copies_1d(gy, d.N, d.nely, d.py, ey, iy);
    const int mz = gs_copies_1d(gz, d.N, d.nelz, d.pz, ez, iz);
    const int64_t n3 = (int64_t)d.n * d.n * d.n;
    R.m = 0;
    for (int c = 0; c < mz; ++c)
        for (int b = 0; b < my; ++b)
            R.off[R.m++] = ((int64_t)ey[b] + (int64_t)d.nely * ez[c]) * d.nelx * n3 +
                           (int64_t)(iz[c] * d.n + iy[b]) * d.n;
}

// Copy k (y/z part) x a (x part) of a unique node; valid when k < R.m, a < mx.
#define UQ_FOR_COPIES(R, mx, xo, BODY)                              \
    _Pragma("unroll") for (int k_ = 0; k_ < 4; ++k_)                \
        _Pragma("unroll") for (int a_ = 0; a_ < 2; ++a_)            \
            if (k_ < (R).m && a_ < (mx)) {                          \
                const int64_t cp = (R).off[k_] + (xo)[a_];          \
                BODY;                                               \
            }

__device__ __forceinline__ void uniq_item(const ProbDesc &P, const PState &S, int ph, int64_t item,
                                          double v[3])
{
    const GsDesc &d = P.gs;
    const int nxch = (d.ngx + SEM_SOLVE_THREADS - 1) / SEM_SOLVE_THREADS;
    const int it32 = (int)item;  // unique-node items fit in 32 bits (checked at setup)
    const int rg = it32 / nxch;
    const int gx = (it32 - rg * nxch) * SEM_SOLVE_THREADS + threadIdx.x;
    const int rows = d.ngy * d.ngz;
    if (gx >= d.ngx) return;
    const int64_t n3 = (int64_t)d.n * d.n * d.n;
    int ex[2], ix[2];
    const int mx = gs_copies_1d(gx, d.N, d.nelx, d.px, ex, ix);
    const int64_t xo[2] = {ex[0] * n3 + ix[0], mx > 1 ? ex[1] * n3 + ix[1] : 0};
    constexpr int RU = SEM_UQ_ROWS;
    RowCopies R[RU];
    bool ok[RU];
#pragma unroll
    for (int r = 0; r < RU; ++r) {
        const int row = rg * RU + r;
        ok[r] = row < rows;
        if (ok[r]) row_copies(d, row, R[r]);
        else R[r].m = 0;
    }
    switch (ph) {
        case PH_JACGS: {
            if (P.jac_cached) {  // the Jacobi inverse is kept from an earlier solve: only sum b
#pragma unroll
                for (int r = 0; r < RU; ++r)
                    if (ok[r]) v[0] += __ldcg(P.b + R[r].off[0] + xo[0]);
                break;
            }
            double s[RU], bv[RU];
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                s[r] = 0.0;
                bv[r] = 0.0;
                if (!ok[r]) continue;
                UQ_FOR_COPIES(R[r], mx, xo, s[r] += __ldcg(P.minv + cp));
                bv[r] = __ldcg(P.b + R[r].off[0] + xo[0]);
            }
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                if (!ok[r]) continue;
                const double rinv = 1.0 / s[r];
                UQ_FOR_COPIES(R[r], mx, xo, {
                    P.minv[cp] = rinv;
                    if (P.minv32) P.minv32[cp] = (float)rinv;
                });
                v[0] += bv[r];
            }
        } break;
        case PH_R0:
        case PH_R64: {
            double s[RU], bv[RU], mv[RU];
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                s[r] = 0.0;
                bv[r] = mv[r] = 0.0;
                if (!ok[r]) continue;
                UQ_FOR_COPIES(R[r], mx, xo, s[r] += __ldcg(P.w + cp));
                const int64_t f = R[r].off[0] + xo[0];
                bv[r] = __ldcg(P.b + f) - S.bmean;
                if (ph == PH_R0) mv[r] = __ldcg(P.minv + f);
            }
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                if (!ok[r]) continue;
                const double rv = bv[r] - s[r];
                UQ_FOR_COPIES(R[r], mx, xo, P.r[cp] = rv);
                v[0] = fma(rv, rv, v[0]);
                if (ph == PH_R0) {
                    v[1] = fma(rv, mv[r] * rv, v[1]);
                    v[2] = fma(bv[r], bv[r], v[2]);
                } else {
                    v[1] = fma(bv[r], bv[r], v[1]);
                }
            }
        } break;
        case PH_C: {
            double s[RU], r0[RU], mv[RU];
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                s[r] = r0[r] = mv[r] = 0.0;
                if (!ok[r]) continue;
                UQ_FOR_COPIES(R[r], mx, xo, s[r] += __ldcg(P.w + cp));
                const int64_t f = R[r].off[0] + xo[0];
                r0[r] = __ldcg(P.r + f);
                mv[r] = __ldcg(P.minv + f);
            }
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                if (!ok[r]) continue;
                const double rv = r0[r] - S.alpha * s[r];
                UQ_FOR_COPIES(R[r], mx, xo, P.r[cp] = rv);
                v[0] = fma(rv, rv, v[0]);
                v[1] = fma(rv, mv[r] * rv, v[1]);
            }
        } break;
        case PH_INIT32: {
            double r0[RU];
            float mv[RU];
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                r0[r] = 0.0;
                mv[r] = 0.f;
                if (!ok[r]) continue;
                const int64_t f = R[r].off[0] + xo[0];
                r0[r] = __ldcg(P.r + f);
                mv[r] = __ldcg(P.minv32 + f);
            }
            dfacc d0 = {0.f, 0.f}, d1 = {0.f, 0.f};
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                if (!ok[r]) continue;
                const float rv = (float)(r0[r] / S.scale);
                UQ_FOR_COPIES(R[r], mx, xo, {
                    P.r32[cp] = rv;
                    P.d32[cp] = 0.0f;
                });
                dot2_acc(d0, rv, rv);
                dot2_acc(d1, rv, mv[r] * rv);
            }
            v[0] += dfacc_value(d0);
            v[1] += dfacc_value(d1);
        } break;
        case PH_C32: {
            float s[RU], r0[RU], mv[RU];
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                s[r] = r0[r] = mv[r] = 0.f;
                if (!ok[r]) continue;
                UQ_FOR_COPIES(R[r], mx, xo, s[r] += __ldcg(P.w32 + cp));
                const int64_t f = R[r].off[0] + xo[0];
                r0[r] = __ldcg(P.r32 + f);
                mv[r] = __ldcg(P.minv32 + f);
            }
            const float a = (float)S.alpha;
            dfacc d0 = {0.f, 0.f}, d1 = {0.f, 0.f};
#pragma unroll
            for (int r = 0; r < RU; ++r) {
                if (!ok[r]) continue;
                const float rv = r0[r] - a * s[r];
                UQ_FOR_COPIES(R[r], mx, xo, P.r32[cp] = rv);
                dot2_acc(d0, rv, rv);
                dot2_acc(d1, rv, mv[r] * rv);
            }
            v[0] += dfacc_value(d0);
            v[1] += dfacc_value(d1);
        } break;
        default: break;
    }
}

__device__ __forceinline__ void local_item(const ProbDesc &P, const PState &S, int ph, int64_t chunk,
                                           double v[3])
{
    const int64_t q = chunk * SEM_SOLVE_THREADS + threadIdx.x;
    if (q >= P.nL) return;
    const int n = P.n, n3 = n * n * n;
    const int64_t e = q / n3;
    const int l = (int)(q - e * n3);
    switch (ph) {
        case PH_JAC: {
            const int i = l % n, j = (l / n) % n, k = l / (n * n);
            const double *g = P.geo64 + e * 7 * n3;
            const double *D = P.D64;
            double s = 0.0;
            for (int t = 0; t < n; ++t) {
                const double a = D[t * n + i], b = D[t * n + j], c = D[t * n + k];
                s += a * a * g[0 * n3 + (k * n + j) * n + t];
                s += b * b * g[1 * n3 + (k * n + t) * n + i];
                s += c * c * g[2 * n3 + (t * n + j) * n + i];
            }
            const double di = D[i * n + i], dj = D[j * n + j], dk = D[k * n + k];
            s += 2.0 * (di * dj * g[3 * n3 + l] + di * dk * g[4 * n3 + l] + dj * dk * g[5 * n3 + l]);
            P.minv[q] = P.h1 * s + P.h2 * g[6 * n3 + l];
        } break;
        case PH_UPD: {
            // the FP64 p vector is unused by refinement: it keeps x until the
            // next residual accepts the step
            float dv = __ldcg(P.d32 + q);
            if (S.pending) dv = fmaf((float)S.alpha, __ldcg(P.p32 + q), dv);
            const double xo = __ldcg(P.x + q);
            P.p[q] = xo;
            P.x[q] = fma(S.scale, (double)dv, xo);
        } break;
        case PH_XREST:
            P.x[q] = __ldcg(P.p + q);
            break;
        case PH_XUPD:
            P.x[q] = fma(S.alpha, __ldcg(P.p + q), __ldcg(P.x + q));
            break;
        case PH_FINAL:
            v[0] = fma(P.geo64[(e * 7 + 6) * n3 + l], __ldcg(P.x + q), v[0]);
            break;
        case PH_SHIFT:
            P.x[q] = __ldcg(P.x + q) - S.shift;
            break;
        default: break;
    }
}

// ---------------------------------------------------------------------------
// per-problem state machine (run by one thread of the last CTA of a step)
// ---------------------------------------------------------------------------

template <int MAXP>
__device__ void advance(const SolveParams<MAXP> &prm, const ProbDesc &P, PState &S, const double *red)
{
    const int ph = S.phase;
    auto finish = [&](int status) {
        S.status = status;
        S.phase = P.singular ? PH_FINAL : PH_DONE;
    };
    // after a C phase the last alpha p is not yet in x
    auto finish_pending = [&](int status) {
        S.status = status;
        S.phase = PH_XUPD;
    };
    switch (ph) {
        case PH_JAC: S.phase = PH_JACGS; break;
        case PH_JACGS:
            S.bmean = P.singular ? red[0] / (double)P.nG : 0.0;
            S.phase = PH_AX0;
            break;
        case PH_AX0: S.phase = prm.mixed ? PH_R64 : PH_R0; break;
        case PH_R0: {
            S.bnorm = sqrt(red[2]);
            S.rnorm = sqrt(red[0]);
            S.target = prm.abs_tol ? prm.tol : prm.tol * S.bnorm;
            if (!isfinite(S.rnorm) || !isfinite(S.bnorm)) { finish(SEM_ERR_BREAKDOWN); break; }
            if (S.rnorm <= S.target) { finish(SEM_OK); break; }
            if (prm.maxit <= 0) { finish(SEM_ERR_NOT_CONVERGED); break; }
            S.rz = red[1];
            S.first = 1;
            S.beta = 0.0;
            S.phase = PH_A;
        } break;
        case PH_A: {
            const double pw = red[0];
            if (!(pw > 0.0) || !isfinite(pw)) { finish(SEM_ERR_BREAKDOWN); break; }
            S.alpha = S.rz / pw;
            S.phase = PH_C;
        } break;
        case PH_C: {
            S.iters += 1;
            S.rnorm = sqrt(red[0]);
            if (!isfinite(S.rnorm)) { finish_pending(SEM_ERR_BREAKDOWN); break; }
            if (S.rnorm <= S.target) { finish_pending(SEM_OK); break; }
            if (S.iters >= prm.maxit) { finish_pending(SEM_ERR_NOT_CONVERGED); break; }
            S.beta = red[1] / S.rz;
            S.rz = red[1];
            S.first = 0;
            S.phase = PH_A;
        } break;
        case PH_R64: {
            const double rn = sqrt(red[0]);
            if (S.outer == 0) {
                S.bnorm = sqrt(red[1]);
                S.target = prm.abs_tol ? prm.tol : prm.tol * S.bnorm;
            }
            if (rn <= S.target) { S.rnorm = rn; finish(SEM_OK); break; }
            // a step that did not lower the FP64 residual (or made it non-finite)
            // is undone: x returns to the iterate before it
            if (S.outer > 0 && !(rn <= S.prev_rnorm)) {
                S.rnorm = S.prev_rnorm;
                S.status = SEM_ERR_NOT_CONVERGED;
                S.phase = PH_XREST;
                break;
            }
            S.rnorm = rn;
            if (!isfinite(rn) || !isfinite(S.bnorm)) { finish(SEM_ERR_BREAKDOWN); break; }
            if (S.outer >= prm.max_outer || S.iters >= prm.maxit) { finish(SEM_ERR_NOT_CONVERGED); break; }
            if (S.outer > 0 && rn > 0.5 * S.prev_rnorm) { finish(SEM_ERR_NOT_CONVERGED); break; }
            S.prev_rnorm = rn;
            S.scale = rn;
            S.phase = PH_INIT32;
        } break;
        case PH_INIT32: {
            // the inner solve needs to reduce its residual only as far as the
            // outer target requires (with a factor 2 margin), never further
            // than inner_tol
            double rel = 0.5 * S.target / S.rnorm;
            if (rel < prm.inner_tol) rel = prm.inner_tol;
            if (rel > 0.5) rel = 0.5;
            S.inner_target = rel * sqrt(red[0]);
            S.rz = red[1];
            S.first = 1;
            S.beta = 0.0;
            S.inner_iters = 0;
            S.pending = 0;
            S.phase = (red[0] > 0.0) ? PH_A32 : PH_UPD;
        } break;
        case PH_A32: {
            const double pw = red[0];
            if (!(pw > 0.0) || !isfinite(pw)) { S.pending = 0; S.phase = PH_UPD; break; }
            S.alpha = S.rz / pw;
            S.phase = PH_C32;
        } break;
        case PH_C32: {
            S.iters += 1;
            S.inner_iters += 1;
            const double rn = sqrt(red[0]);
            if (!isfinite(rn) || rn <= S.inner_target || S.iters >= prm.maxit) {
                S.pending = 1;
                S.phase = PH_UPD;
                break;
            }
            S.beta = red[1] / S.rz;
            S.rz = red[1];
            S.first = 0;
            S.phase = PH_A32;
        } break;
        case PH_UPD: S.outer += 1; S.phase = PH_AX0; break;
        case PH_FINAL: S.shift = red[0] / P.volume; S.phase = PH_SHIFT; break;
        case PH_SHIFT: S.phase = PH_DONE; break;
        case PH_XUPD: case PH_XREST: S.phase = P.singular ? PH_FINAL : PH_DONE; break;
        default: S.phase = PH_DONE; break;
    }
    S.nvals = phase_nvals(S.phase);
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

template <int MAXP, int MODE, int... NPs>
__global__ void __launch_bounds__(SEM_SOLVE_THREADS, MODE == MODE_F32 ? SEM_SOLVE_F32_MINB : SEM_SOLVE_F64_MINB)
    k_solve(const __grid_constant__ SolveParams<MAXP> prm)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_part[MAXP][3];
    __shared__ double s_red[SEM_SOLVE_THREADS / 32 * 3];
    __shared__ int s_phase[MAXP];
    __shared__ long long s_offs[MAXP + 1];
    __shared__ double s_alpha[MAXP], s_beta[MAXP], s_bmean[MAXP], s_scale[MAXP], s_shift[MAXP];
    __shared__ int s_first[MAXP], s_pending[MAXP];
    __shared__ int s_last, s_stop;
    __shared__ unsigned s_gen;
    const int np = prm.nprob;
    SyncState *sync = prm.sync;
    if constexpr (MODE == MODE_F64)  // reduction words of the block-floating-point element phases
        for (int t = threadIdx.x; t < SEM_BFP_RED_BYTES / 4; t += blockDim.x)
            reinterpret_cast<unsigned *>(smem)[t] = 0u;

    for (int step = 0;; ++step) {
        // ---- schedule of this step
        if (threadIdx.x == 0) {
            long long o = 0;
            for (int p = 0; p < np; ++p) {
                int ph;
                if (step == 0) {
                    ph = prm.prob[p].jac_cached ? PH_JACGS : PH_JAC;
                } else {
                    ph = ((volatile int *)prm.sched)[p];
                }
                s_phase[p] = ph;
                s_offs[p] = o;
                o += phase_items(prm.prob[p], ph);
            }
            s_offs[np] = o;
            s_stop = (step > 0 && ((volatile int *)&sync->finished)[0]) ||
                     ((volatile int *)&sync->err)[0];
        }
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            const volatile PState *S = prm.st + p;
            s_alpha[p] = S->alpha;
            s_beta[p] = S->beta;
            s_bmean[p] = S->bmean;
            s_scale[p] = S->scale;
            s_shift[p] = S->shift;
            s_first[p] = S->first;
            s_pending[p] = S->pending;
            s_part[p][0] = s_part[p][1] = s_part[p][2] = 0.0;
        }
        __syncthreads();
        if (s_stop) break;

        // ---- work items
        const long long total = s_offs[np];
        double v[3] = {0.0, 0.0, 0.0};
        double acc = 0.0;
        int cur = -1;
        for (long long it = blockIdx.x; it < total; it += gridDim.x) {
            int p = 0;
            while (p + 1 < np && s_offs[p + 1] <= it) ++p;
            if (p != cur) {
                if (cur >= 0) {
                    v[0] += acc;
                    acc = 0.0;
                    block_accumulate(v, s_red, s_part[cur]);
                }
                cur = p;
            }
            const ProbDesc &P = prm.prob[p];
            const int ph = s_phase[p];
            const int64_t local = it - s_offs[p];
            PState S;
            S.alpha = s_alpha[p];
            S.beta = s_beta[p];
            S.bmean = s_bmean[p];
            S.scale = s_scale[p];
            S.shift = s_shift[p];
            S.pending = s_pending[p];
            if (ph == PH_AX0 || ph == PH_A || ph == PH_A32) {
                ElemDispatch<MODE, NPs...>::run(P, ph, S.alpha, S.beta, s_first[p], local,
                                                prm.inner_tc, smem, acc);
            } else if (ph == PH_JAC || ph == PH_UPD || ph == PH_FINAL || ph == PH_SHIFT ||
                       ph == PH_XUPD || ph == PH_XREST) {
                local_item(P, S, ph, local, v);
            } else {
                uniq_item(P, S, ph, local, v);
            }
        }
        if (cur >= 0) {
            v[0] += acc;
            block_accumulate(v, s_red, s_part[cur]);
        }

        // ---- publish partials, reducing barrier
        double *part = prm.partials + (size_t)blockIdx.x * MAXP * 3;
        for (int t = threadIdx.x; t < np * 3; t += blockDim.x) part[t] = s_part[t / 3][t % 3];
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_gen = ((volatile unsigned *)&sync->gen)[0];
            const unsigned arrived = atomicAdd(&sync->count, 1u);
            s_last = (arrived == gridDim.x - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            // fixed-order reduction of every (problem, value) pair: one warp each
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int pk = warp; pk < np * 3; pk += SEM_SOLVE_THREADS / 32) {
                const int p = pk / 3, k = pk % 3;
                double s = 0.0;
                if (k < phase_nvals(s_phase[p]))
                    for (int b = lane; b < (int)gridDim.x; b += 32)
                        s += __ldcg(prm.partials + ((size_t)b * MAXP + p) * 3 + k);
                s = warp_sum(s);
                if (lane == 0) s_part[p][k] = s;
            }
            __syncthreads();
            for (int p = threadIdx.x; p < np; p += blockDim.x) {
                PState S = prm.st[p];
                S.phase = s_phase[p];
                advance<MAXP>(prm, prm.prob[p], S, s_part[p]);
                prm.st[p] = S;
                prm.sched[p] = S.phase;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int fin = 1;
                for (int p = 0; p < np; ++p) fin &= (prm.sched[p] == PH_DONE);
                sync->finished = fin;
                sync->count = 0;
                __threadfence();
                atomicAdd(&sync->gen, 1u);
            }
        } else if (threadIdx.x == 0) {
            const unsigned long long t0 = sem_globaltimer();
            while (ld_acquire_u32(&sync->gen) == s_gen) {
                if (((volatile int *)&sync->err)[0]) break;
                if ((long long)(sem_globaltimer() - t0) > prm.timeout_ns) {
                    atomicExch(&sync->err, SEM_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        __syncthreads();
    }
}

constexpr size_t sem_max_sz(size_t a, size_t b) { return a > b ? a : b; }

// Dynamic shared memory of the element phases of one problem order and mode.
template <int NP, int MODE>
constexpr size_t solve_smem_np()
{
    return MODE == MODE_F64N ? ax_smem_bytes<NP, double>()
           : MODE == MODE_F64 ? (solve_bfp<NP>() ? SEM_BFP_RED_BYTES + ax_bfp_smem_bytes_ne<NP, BfpCfg<NP>::NE>()
                                 : df_folded<NP>() ? ax_dfeo_smem_bytes<NP>() : ax_df_smem_bytes<NP>())
           : MODE == MODE_F32 ? sem_max_sz(ax_smem_bytes<NP, float>(), ax_df_lowreg_smem_bytes<NP>())
                              : sem_max_sz(sem_max_sz(ax_tc_smem_bytes<NP>(), ax_tc_split_smem_bytes<NP>()),
                                           sem_max_sz(ax_df_lowreg_smem_bytes<NP>(), ax_smem_bytes<NP, float>()));
}

template <int MODE, int... NPs>
struct SmemMax;
template <int MODE>
struct SmemMax<MODE> {
    static constexpr size_t v = 0;
};
template <int MODE, int NP0, int... NPs>
struct SmemMax<MODE, NP0, NPs...> {
    static constexpr size_t v = sem_max_sz(solve_smem_np<NP0, MODE>(), SmemMax<MODE, NPs...>::v);
};

// Host launcher (cooperative, grid sized for co-residency).
template <int MAXP, int MODE, int... NPs>
int launch_solve(const SolveParams<MAXP> &prm, int num_sms, long long max_items, cudaStream_t s)
{
    auto kern = k_solve<MAXP, MODE, NPs...>;
    const size_t smem = SmemMax<MODE, NPs...>::v;
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(kern, smem, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SEM_SOLVE_THREADS, smem));
    if (per_sm < 1) return SEM_ERR_ARG;
    long long grid = (long long)per_sm * num_sms;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    void *args[] = {(void *)&prm};
    SEM_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)grid),
                                         dim3(SEM_SOLVE_THREADS), args, smem, s));
    return SEM_OK;
}

// Maximum grid the solver may use (sizes the partials buffer).
#define SEM_SOLVE_MAX_GRID_PER_SM 8
