// ax_df.cu -- stand-alone FP64-accurate sem_ax on the FP32 pipes (float pairs).
#include <math.h>
#include <stdlib.h>

#include "ax_bfp.cuh"
#include "ax_df.cuh"
#include "ax_dfeo.cuh"
#include "common.cuh"
#include "tma.cuh"

// Thread 0 asks L2 for the geometry of this block's current element group
// (read after the gradient stage, about half a group later) and for the u of
// its next group (read at that group's start).  Elements are clipped to E.
// Prefetching the next group's geometry as well (a whole group ahead) was
// slower (0.468 vs 0.427 ms at 32^3, N=7) and L2 evicted a third of those
// lines before use (37% more DRAM reads).  u == nullptr skips the u prefetch
// (u in mapped host memory, read over the host link by the loads themselves).
template <int NP>
__device__ __forceinline__ void df_prefetch(const double *u, const dfp *geo, int64_t e0, int64_t en,
                                            int ne, int64_t E)
{
    constexpr int64_t NP3 = NP * NP * NP;
    if (threadIdx.x != 0) return;
    if (e0 < E) l2_prefetch_span(geo, e0 * 7 * NP3 * 8, (e0 + ne < E ? e0 + ne : E) * 7 * NP3 * 8);
    if (u && en < E) l2_prefetch_span(u, en * NP3 * 8, (en + ne < E ? en + ne : E) * NP3 * 8);
}

template <int NP>
__global__ void __launch_bounds__(AxDfCfg<NP>::THREADS, 2)
    k_ax_df(const double *__restrict__ u, double *__restrict__ w, const dfp *__restrict__ geo,
            const dfp *__restrict__ D, dfp h1, dfp h2, int64_t E, const double *upf)
{
    using C = AxDfCfg<NP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dfp *sm = reinterpret_cast<dfp *>(smem_raw);
    dfp *sD = sm, *sDT = sm + NP * NP;
    int *sexp = reinterpret_cast<int *>(sm + 2 * NP * NP + (size_t)C::NE * 3 * C::NP3);
    const int grp = threadIdx.x / C::NP2, tid = threadIdx.x - grp * C::NP2;
    dfp *su = sm + 2 * NP * NP + (size_t)grp * 3 * C::NP3;
    dfp *svr = su + C::NP3, *svs = svr + C::NP3;
    ax_df_load_D<NP>(D, sD, sDT);
    for (int64_t e0 = (int64_t)blockIdx.x * C::NE; e0 < E; e0 += (int64_t)gridDim.x * C::NE) {
        df_prefetch<NP>(upf, geo, e0, e0 + (int64_t)gridDim.x * C::NE, C::NE, E);
        const int64_t e = e0 + grp;
        const bool active = e < E;
        const int64_t off = (active ? e : 0) * C::NP3;
        const double *ue = u + off;
        double *we = w + off;
        auto load = [&](int p) { return ue[p]; };
        auto store = [&](int p, double v) { we[p] = v; };
        ax_df_element<NP>(load, store, geo + (active ? e : 0) * 7 * C::NP3, h1, h2, sD, sDT, su, svr,
                          svs, sexp + grp, tid, active);
    }
}

// Folded (even-odd) variant for even NP, NE elements per block.  Each block is
// resident on the SM with at most 128 registers a thread (blocks of
// 32 ceil(T/32) threads, 512 per SM at that register count).
template <int NP, int NE>
struct DfeoShape {
    static constexpr int THREADS = NE * NP * NP;
    static constexpr int MINB = 16 / ((THREADS + 31) / 32) > 0 ? 16 / ((THREADS + 31) / 32) : 1;
};

template <int NP, int NE, int GS>
__global__ void __launch_bounds__(DfeoShape<NP, NE>::THREADS, DfeoShape<NP, NE>::MINB)
    k_ax_dfeo(const double *__restrict__ u, double *__restrict__ w, const dfp *__restrict__ geo,
              const dfp *__restrict__ tabs, dfp h1, dfp h2, int64_t E, const double *upf)
{
    using C = AxEoCfg<NP>;
    constexpr int HH = (NP / 2) * (NP / 2);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dfp *sm = reinterpret_cast<dfp *>(smem_raw);
    dfp *stab = sm;
    int *sexp = reinterpret_cast<int *>(sm + 4 * HH + (size_t)NE * 5 * C::SLAB);
    const int grp = threadIdx.x / C::NP2, tid = threadIdx.x - grp * C::NP2;
    dfp *slab = sm + 4 * HH + (size_t)grp * 5 * C::SLAB;
    for (int t = threadIdx.x; t < 4 * HH; t += blockDim.x) stab[t] = tabs[t];
    // with block barriers the element's first barrier publishes the tables
    if constexpr (GS != 0) __syncthreads();
    for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < E; e0 += (int64_t)gridDim.x * NE) {
        df_prefetch<NP>(upf, geo, e0, e0 + (int64_t)gridDim.x * NE, NE, E);
        const int64_t e = e0 + grp;
        const bool active = e < E;
        const int64_t off = (active ? e : 0) * C::NP3;
        const double *ue = u + off;
        double *we = w + off;
        auto load = [&](int p) { return ue[p]; };
        auto store = [&](int p, double v) { we[p] = v; };
        ax_dfeo_element<NP, GS>(load, store, geo + (active ? e : 0) * 7 * C::NP3, h1, h2, stab, slab,
                                sexp + grp, tid, active, grp);
    }
}

template <int NP, int NE, int GS>
static int launch_dfeo(const sem_ctx *c, const double *u, double *w, dfp H1, dfp H2, cudaStream_t s)
{
    constexpr int T = DfeoShape<NP, NE>::THREADS;
    const size_t smem = ax_dfeo_smem_bytes_ne<NP, NE>();
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(k_ax_dfeo<NP, NE, GS>, smem, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_dfeo<NP, NE, GS>, T, smem));
    if (per_sm < 1) return SEM_ERR_ARG;
    int64_t groups = sem_ceil_div(c->E, NE);
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > groups) grid = groups;
    k_ax_dfeo<NP, NE, GS><<<(unsigned)grid, T, smem, s>>>(u, w, (const dfp *)c->geodf,
                                                      (const dfp *)c->tabdfeo, H1, H2, c->E,
                                                      c->u_sysmem ? nullptr : u);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

// Tile-shape candidates of the folded kernel (N+1 <= 10): 0 = AxEoCfg's
// elements per block (256 threads at most) with block barriers; 1 = the same
// with one named barrier per element group where a group is whole warps
// ((N+1)^2 a multiple of 32, 2..15 groups), else as 0; 2 = half the elements
// per block.
template <int NP>
constexpr int dfeo_ne(int variant)
{
    constexpr int NE0 = AxEoCfg<NP>::NE;
    const int ne = variant == 2 ? NE0 / 2 : NE0;
    return NP > 10 || ne < 1 ? NE0 : ne;
}

template <int NP>
constexpr int dfeo_group_sync()
{
    constexpr int NE0 = AxEoCfg<NP>::NE;
    return (NP * NP) % 32 == 0 && NE0 >= 2 && NE0 <= 15 && NP <= 10 ? NP * NP : 0;
}

int sem_launch_ax_bfp(const sem_ctx *c, int variant, const double *u, double *w, double h1,
                      double h2, cudaStream_t s);  // ax_bfp.cu

template <int NP>
static int launch_df(const sem_ctx *c, const double *u, double *w, double h1, double h2,
                     cudaStream_t s)
{
    if (sem_ax_variant(c->N, SEM_F64) >= 3) {
        const int rc = sem_launch_ax_bfp(c, sem_ax_variant(c->N, SEM_F64), u, w, h1, h2, s);
        if (rc != SEM_ERR_ARG) return rc;  // else the order has no block-floating-point kernel
    }
    if constexpr (AxEoCfg<NP>::OK) {
        if (ax_dfeo_smem_bytes<NP>() <= 227 * 1024) {
            const float a = (float)h1, b = (float)h2;
            const dfp H1 = {a, (float)(h1 - (double)a)}, H2 = {b, (float)(h2 - (double)b)};
            const int v = sem_ax_variant(c->N, SEM_F64);
            constexpr int NE0 = AxEoCfg<NP>::NE, N2 = dfeo_ne<NP>(2), GS = dfeo_group_sync<NP>();
            if (v == 1 && GS) return launch_dfeo<NP, NE0, GS>(c, u, w, H1, H2, s);
            if (v == 2 && N2 != NE0) return launch_dfeo<NP, N2, 0>(c, u, w, H1, H2, s);
            return launch_dfeo<NP, NE0, 0>(c, u, w, H1, H2, s);
        }
    }
    using C = AxDfCfg<NP>;
    const size_t smem = ax_df_smem_bytes<NP>();
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(k_ax_df<NP>, smem, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_df<NP>, C::THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t groups = sem_ceil_div(c->E, C::NE);
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > groups) grid = groups;
    const float h1h = (float)h1, h2h = (float)h2;
    const dfp H1 = {h1h, (float)(h1 - (double)h1h)}, H2 = {h2h, (float)(h2 - (double)h2h)};
    k_ax_df<NP><<<(unsigned)grid, C::THREADS, smem, s>>>(u, w, (const dfp *)c->geodf,
                                                        (const dfp *)c->tabdf, H1, H2, c->E,
                                                        c->u_sysmem ? nullptr : u);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

int sem_launch_ax_df(const sem_ctx *c, const double *u, double *w, double h1, double h2,
                     cudaStream_t s)
{
    SEM_DISPATCH_NP(c->n, return launch_df<NP>(c, u, w, h1, h2, s));
    return SEM_ERR_ARG;
}

// Float-pair copy of the FP64 geometry (hi = round(g), lo = round(g - hi)).
__global__ void k_split_geo(const double *__restrict__ g64, dfp *__restrict__ gdf, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double g = g64[t];
    const float h = __double2float_rn(g);
    gdf[t] = {h, __double2float_rn(g - (double)h)};
}

int sem_make_geo_df(sem_ctx *c)
{
    const int64_t n = 7 * c->nL;
    SEM_CUDA(cudaMalloc(&c->geodf, sizeof(dfp) * n));
    k_split_geo<<<(unsigned)sem_ceil_div(n, 256), 256>>>(c->geo64, (dfp *)c->geodf, n);
    SEM_CHECK_LAUNCH();
    if (c->n % 2 == 0) {  // tables of the block-floating-point kernel
        BfpTabs *T = (BfpTabs *)calloc(1, sizeof(BfpTabs));
        if (!T) return SEM_ERR_NOMEM;
        ax_bfp_tables(c->n, c->hD, T);
        c->bfp_tabs = T;
    }
    dfp hD[SEM_NPMAX * SEM_NPMAX];
    for (int t = 0; t < c->n * c->n; ++t) {
        const float h = (float)c->hD[t];
        hD[t] = {h, (float)(c->hD[t] - (double)h)};
    }
    SEM_CUDA(cudaMalloc(&c->tabdf, sizeof(dfp) * c->n * c->n));
    SEM_CUDA(cudaMemcpy(c->tabdf, hD, sizeof(dfp) * c->n * c->n, cudaMemcpyHostToDevice));
    if (c->n % 2 == 0) {  // half tables of the folded operator
        dfp ht[4 * (SEM_NPMAX / 2) * (SEM_NPMAX / 2)];
        ax_dfeo_tables(c->n, c->hD, ht);
        const size_t nb = sizeof(dfp) * 4 * (c->n / 2) * (c->n / 2);
        SEM_CUDA(cudaMalloc(&c->tabdfeo, nb));
        SEM_CUDA(cudaMemcpy(c->tabdfeo, ht, nb, cudaMemcpyHostToDevice));
    }
    return SEM_OK;
}
