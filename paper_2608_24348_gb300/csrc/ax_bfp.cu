// ax_bfp.cu -- stand-alone FP64-accurate sem_ax with block-floating-point
// pairs (ax_bfp.cuh): direct loads, or u staged by bulk copies; scalar or
// paired FP32 instructions.  Instantiated for even N+1 <= 12 (larger orders
// exceed the register budget of two 256-thread blocks per SM).
#include <stdint.h>

#include "ax_bfp.cuh"
#include "tma.cuh"

// Thread 0 asks L2 for the geometry of this block's current element group
// (read after the gradient stage) and, unless u is null, for the u of its next
// group.  Elements are clipped to E.
template <int NP>
__device__ __forceinline__ void bfp_prefetch(const double *u, const dfp *geo, int64_t e0, int64_t en,
                                             int ne, int64_t E)
{
    constexpr int64_t NP3 = NP * NP * NP;
    if (threadIdx.x != 0) return;
    if (e0 < E) l2_prefetch_span(geo, e0 * 7 * NP3 * 8, (e0 + ne < E ? e0 + ne : E) * 7 * NP3 * 8);
    if (u && en < E) l2_prefetch_span(u, en * NP3 * 8, (en + ne < E ? en + ne : E) * NP3 * 8);
}

// Block-floating-point variant (ax_bfp.cuh) for even NP: NE elements per block
// of at most 256 threads, two blocks per SM (128 registers a thread).
template <int NP, bool PAIR>
__global__ void __launch_bounds__(BfpCfg<NP>::THREADS, 2)
    k_ax_bfp(const double *__restrict__ u, double *__restrict__ w, const dfp *__restrict__ geo,
             const __grid_constant__ BfpTabs T, dfp h1, dfp h2, int64_t E, const double *upf)
{
    using C = BfpCfg<NP>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    dfp *slabs = reinterpret_cast<dfp *>(smem_raw);
    unsigned *red = reinterpret_cast<unsigned *>(slabs + (size_t)C::NE * 3 * C::SLAB);
    const int grp = threadIdx.x / C::NP2, tid = threadIdx.x - grp * C::NP2;
    for (int t = threadIdx.x; t < 8 * C::NE; t += blockDim.x) red[t] = 0u;
    __syncthreads();
    for (int64_t e0 = (int64_t)blockIdx.x * C::NE; e0 < E; e0 += (int64_t)gridDim.x * C::NE) {
        bfp_prefetch<NP>(upf, geo, e0, e0 + (int64_t)gridDim.x * C::NE, C::NE, E);
        const int64_t e = e0 + grp;
        const bool active = e < E;
        const int64_t off = (active ? e : 0) * C::NP3;
        const double *ue = u + off;
        double *we = w + off;
        auto load = [&](int p) { return ue[p]; };
        auto store = [&](int p, double v) { we[p] = v; };
        ax_bfp_element<NP, PAIR>(load, store, geo + (active ? e : 0) * 7 * C::NP3, h1, h2, T,
                                 slabs + (size_t)grp * 3 * C::SLAB, red + grp * 8, tid, active,
                                 [] {});
    }
}

// The same with each element group's u (one contiguous block of NE NP^3
// doubles) copied into shared memory by a bulk copy (cp.async.bulk, mbarrier
// completion) issued one group ahead: the copy of group g+1 starts as soon as
// every thread has read group g's u, so the operator never waits on u in
// global memory.  Every wait is bounded; a wait that runs out records
// SEM_ERR_TIMEOUT in err, the block waits (bounded) for its copy in flight
// and stops.
template <int NP, int NEB, int WARPS_SM = 16>
struct BfpStage {
    using C = BfpCfg<NP>;
    static constexpr int NE = NEB;
    static constexpr int THREADS = NEB * C::NP2;
    // resident blocks per SM for WARPS_SM warps (the register budget follows)
    static constexpr int MINB = 32 * WARPS_SM / THREADS > 0 ? 32 * WARPS_SM / THREADS : 1;
    static constexpr size_t U_OFF = (ax_bfp_smem_bytes_ne<NP, NEB>() + 127) / 128 * 128;
    static constexpr size_t U_BYTES = sizeof(double) * NEB * C::NP3;
    static constexpr size_t BAR_OFF = U_OFF + U_BYTES;
    static constexpr size_t SMEM = BAR_OFF + 16;
};

template <int NP, bool PAIR, int NEB, int WSM>
__global__ void __launch_bounds__(BfpStage<NP, NEB, WSM>::THREADS, BfpStage<NP, NEB, WSM>::MINB)
    k_ax_bfp_st(const double *__restrict__ u, double *__restrict__ w, const dfp *__restrict__ geo,
                const __grid_constant__ BfpTabs T, dfp h1, dfp h2, int64_t E, int *err,
                long long timeout_ns)
{
    using S = BfpStage<NP, NEB, WSM>;
    using C = S;
    constexpr int NP2 = NP * NP, NP3 = NP2 * NP, SLAB = BfpCfg<NP>::SLAB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    dfp *slabs = reinterpret_cast<dfp *>(smem_raw);
    unsigned *red = reinterpret_cast<unsigned *>(slabs + (size_t)C::NE * 3 * SLAB);
    const double *ubuf = reinterpret_cast<const double *>(smem_raw + S::U_OFF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + S::BAR_OFF);
    const int grp = threadIdx.x / NP2, tid = threadIdx.x - grp * NP2;
    const int64_t groups = (E + C::NE - 1) / C::NE;
    auto issue = [&](int64_t g) {
        const int64_t e0 = g * C::NE;
        const int64_t ne = (E - e0) < C::NE ? (E - e0) : C::NE;
        const uint32_t ub = (uint32_t)(ne * NP3 * sizeof(double));
        mbar_expect_tx(bar, ub);
        bulk_g2s(smem_raw + S::U_OFF, u + e0 * NP3, ub, bar);
    };
    for (int t = threadIdx.x; t < 8 * C::NE; t += blockDim.x) red[t] = 0u;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && (int64_t)blockIdx.x < groups) issue(blockIdx.x);
    int64_t it = 0;
    bool failed = false;
    for (;; ++it) {
        const int64_t g = blockIdx.x + it * gridDim.x;
        if (g >= groups) break;
        const bool ok = mbar_wait_bounded(bar, (uint32_t)(it & 1), timeout_ns);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const int64_t e0 = g * C::NE;
        bfp_prefetch<NP>(nullptr, geo, e0, e0, C::NE, E);
        const int64_t e = e0 + grp;
        const bool active = e < E;
        const double *ue = ubuf + (size_t)grp * NP3;
        double *we = w + (active ? e : 0) * NP3;
        auto load = [&](int p) { return ue[p]; };
        auto store = [&](int p, double v) { we[p] = v; };
        auto next = [&] {
            const int64_t g2 = g + gridDim.x;
            if (threadIdx.x == 0 && g2 < groups) {
                fence_proxy_async_smem();
                issue(g2);
            }
        };
        ax_bfp_element<NP, PAIR>(load, store, geo + (active ? e : 0) * 7 * NP3, h1, h2, T,
                                 slabs + (size_t)grp * 3 * SLAB, red + grp * 8, tid, active, next);
    }
    if (failed && threadIdx.x == 0) {
        atomicExch(err, SEM_ERR_TIMEOUT);
        // the copy of group `it` may still be in flight: wait for it (bounded)
        mbar_wait_bounded(bar, (uint32_t)(it & 1), timeout_ns);
    }
}

template <int NP, bool PAIR>
static int launch_bfp(const sem_ctx *c, const double *u, double *w, dfp H1, dfp H2, cudaStream_t s)
{
    using C = BfpCfg<NP>;
    if (!c->bfp_tabs) return SEM_ERR_ARG;
    const size_t smem = ax_bfp_smem_bytes_ne<NP, C::NE>();
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(k_ax_bfp<NP, PAIR>, smem, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_bfp<NP, PAIR>, C::THREADS, smem));
    if (per_sm < 1) return SEM_ERR_ARG;
    int64_t groups = sem_ceil_div(c->E, C::NE);
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > groups) grid = groups;
    k_ax_bfp<NP, PAIR><<<(unsigned)grid, C::THREADS, smem, s>>>(u, w, (const dfp *)c->geodf,
                                                                *(const BfpTabs *)c->bfp_tabs, H1, H2,
                                                                c->E, c->u_sysmem ? nullptr : u);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

template <int NP, bool PAIR, int NEB, int WSM = 16>
static int launch_bfp_st(const sem_ctx *c, const double *u, double *w, dfp H1, dfp H2, cudaStream_t s)
{
    using S = BfpStage<NP, NEB, WSM>;
    if (!c->bfp_tabs) return SEM_ERR_ARG;
    auto kern = k_ax_bfp_st<NP, PAIR, NEB, WSM>;
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(kern, S::SMEM, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::THREADS, S::SMEM));
    if (per_sm < 1) return SEM_ERR_ARG;
    int64_t groups = sem_ceil_div(c->E, NEB);
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > groups) grid = groups;
    kern<<<(unsigned)grid, S::THREADS, S::SMEM, s>>>(u, w, (const dfp *)c->geodf,
                                                      *(const BfpTabs *)c->bfp_tabs, H1, H2, c->E,
                                                      (int *)c->err_dev, 2000000000LL);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

template <int NP>
static int launch_bfp_any(const sem_ctx *c, int variant, const double *u, double *w, double h1,
                          double h2, cudaStream_t s)
{
    if constexpr (!BfpCfg<NP>::OK || NP > 12) {
        return SEM_ERR_ARG;
    } else {
        if (ax_bfp_smem_bytes_ne<NP, BfpCfg<NP>::NE>() > 227 * 1024) return SEM_ERR_ARG;
        const float a = (float)h1, b = (float)h2;
        const dfp H1 = {a, (float)(h1 - (double)a)}, H2 = {b, (float)(h2 - (double)b)};
        constexpr int NE0 = BfpCfg<NP>::NE;
        const bool pair = variant == 4 || variant == 6;
        // the staged forms read u with bulk copies: device memory with a
        // 16-byte aligned start only
        if (variant >= 5 && !c->u_sysmem && ((uintptr_t)u & 15) == 0 &&
            BfpStage<NP, NE0, 16>::SMEM <= 227 * 1024) {
            if (variant == 7 && NE0 >= 2) return launch_bfp_st<NP, false, NE0 / 2 ? NE0 / 2 : 1>(c, u, w, H1, H2, s);
            if (variant == 8) return launch_bfp_st<NP, false, 1>(c, u, w, H1, H2, s);
            if (variant == 9) return launch_bfp_st<NP, false, 1, 20>(c, u, w, H1, H2, s);
            if (variant == 10) return launch_bfp_st<NP, false, 1, 24>(c, u, w, H1, H2, s);
            return pair ? launch_bfp_st<NP, true, NE0>(c, u, w, H1, H2, s)
                        : launch_bfp_st<NP, false, NE0>(c, u, w, H1, H2, s);
        }
        return pair ? launch_bfp<NP, true>(c, u, w, H1, H2, s) : launch_bfp<NP, false>(c, u, w, H1, H2, s);
    }
}

int sem_launch_ax_bfp(const sem_ctx *c, int variant, const double *u, double *w, double h1,
                      double h2, cudaStream_t s)
{
    switch (c->n) {
        case 2: return launch_bfp_any<2>(c, variant, u, w, h1, h2, s);
        case 4: return launch_bfp_any<4>(c, variant, u, w, h1, h2, s);
        case 6: return launch_bfp_any<6>(c, variant, u, w, h1, h2, s);
        case 8: return launch_bfp_any<8>(c, variant, u, w, h1, h2, s);
        case 10: return launch_bfp_any<10>(c, variant, u, w, h1, h2, s);
        case 12: return launch_bfp_any<12>(c, variant, u, w, h1, h2, s);
        default: return SEM_ERR_ARG;
    }
}
