// ax_tc.cu -- stand-alone sem_ax with BF16 / FP16 tensor-core contractions.
#include "ax_tc.cuh"
#include "common.cuh"

template <int NP>
__global__ void __launch_bounds__(256)
    k_ax_tc(const float *__restrict__ u, float *__restrict__ w, const float *__restrict__ geo,
            const float *__restrict__ D, float h1, float h2, int64_t E, int fp16)
{
    extern __shared__ __align__(16) unsigned char smem[];
    auto load = [&](int64_t q) { return u[q]; };
    auto store = [&](int64_t q, float v, float) { w[q] = v; };
    const int64_t groups = (E + TcCfg<NP>::NE - 1) / TcCfg<NP>::NE;
    for (int64_t g = blockIdx.x; g < groups; g += gridDim.x)
        ax_tc_group<NP>(load, store, geo, D, h1, h2, E, g, fp16, smem);
}

template <int NP>
static int launch_tc(const sem_ctx *c, const float *u, float *w, float h1, float h2, int fp16,
                     cudaStream_t s)
{
    if constexpr (!TcCfg<NP>::OK) {
        return SEM_ERR_ARG;
    } else {
        const size_t smem = ax_tc_smem_bytes<NP>();
        static std::atomic<unsigned> attr{0};
        SEM_CUDA(sem_smem_attr(k_ax_tc<NP>, smem, attr));
        int per_sm = 0;
        SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_tc<NP>, 256, smem));
        if (per_sm < 1) per_sm = 1;
        int64_t groups = sem_ceil_div(c->E, TcCfg<NP>::NE);
        int64_t grid = (int64_t)per_sm * c->num_sms;
        if (grid > groups) grid = groups;
        k_ax_tc<NP><<<(unsigned)grid, 256, smem, s>>>(u, w, c->geo32, c->tab32 + 2 * c->n, h1, h2,
                                                     c->E, fp16);
        SEM_CHECK_LAUNCH();
        return SEM_OK;
    }
}

int sem_ax_tc(sem_ctx *c, const float *u, float *w, double h1, double h2, int fp16, cudaStream_t s)
{
    if (c->n > 10) return SEM_ERR_ARG;
    SEM_DISPATCH_NP(c->n, return launch_tc<NP>(c, u, w, (float)h1, (float)h2, fp16, s));
    return SEM_ERR_ARG;
}

// Split-operand form (SEM_F16X2_TC / SEM_BF16X3_TC), N+1 <= 8.
template <int NP, bool FP16>
__global__ void __launch_bounds__(256)
    k_ax_tc_split(const float *__restrict__ u, float *__restrict__ w, const float *__restrict__ geo,
                  const float *__restrict__ D, float h1, float h2, int64_t E)
{
    extern __shared__ __align__(16) unsigned char smem[];
    auto load = [&](int64_t q) { return u[q]; };
    auto store = [&](int64_t q, float v, float) { w[q] = v; };
    const int64_t groups = (E + TcSplitCfg<NP>::NE - 1) / TcSplitCfg<NP>::NE;
    for (int64_t g = blockIdx.x; g < groups; g += gridDim.x)
        ax_tc_split_group<NP, FP16>(load, store, geo, D, h1, h2, E, g, smem);
}

template <int NP, bool FP16>
static int launch_tc_split(const sem_ctx *c, const float *u, float *w, float h1, float h2, cudaStream_t s)
{
    if constexpr (!TcSplitCfg<NP>::OK) {
        return SEM_ERR_ARG;
    } else {
        const size_t smem = ax_tc_split_smem_bytes<NP>();
        auto kern = k_ax_tc_split<NP, FP16>;
        static std::atomic<unsigned> attr{0};
        SEM_CUDA(sem_smem_attr(kern, smem, attr));
        int per_sm = 0;
        SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
        if (per_sm < 1) per_sm = 1;
        int64_t groups = sem_ceil_div(c->E, TcSplitCfg<NP>::NE);
        int64_t grid = (int64_t)per_sm * c->num_sms;
        if (grid > groups) grid = groups;
        kern<<<(unsigned)grid, 256, smem, s>>>(u, w, c->geo32, c->tab32 + 2 * c->n, h1, h2, c->E);
        SEM_CHECK_LAUNCH();
        return SEM_OK;
    }
}

int sem_ax_tc_split(sem_ctx *c, const float *u, float *w, double h1, double h2, int fp16, cudaStream_t s)
{
    if (c->n > 8) return SEM_ERR_ARG;
    switch (c->n) {
        case 2: return fp16 ? launch_tc_split<2, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<2, false>(c, u, w, (float)h1, (float)h2, s);
        case 3: return fp16 ? launch_tc_split<3, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<3, false>(c, u, w, (float)h1, (float)h2, s);
        case 4: return fp16 ? launch_tc_split<4, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<4, false>(c, u, w, (float)h1, (float)h2, s);
        case 5: return fp16 ? launch_tc_split<5, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<5, false>(c, u, w, (float)h1, (float)h2, s);
        case 6: return fp16 ? launch_tc_split<6, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<6, false>(c, u, w, (float)h1, (float)h2, s);
        case 7: return fp16 ? launch_tc_split<7, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<7, false>(c, u, w, (float)h1, (float)h2, s);
        case 8: return fp16 ? launch_tc_split<8, true>(c, u, w, (float)h1, (float)h2, s) : launch_tc_split<8, false>(c, u, w, (float)h1, (float)h2, s);
        default: return SEM_ERR_ARG;
    }
}
