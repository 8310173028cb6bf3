// ax_f32.cu -- FP32 stand-alone element operator: direct-load kernel and a
// bulk-copy (TMA) staged kernel.
//
// The staged kernel streams each element group's two contiguous blocks -- the
// u slab (NE (N+1)^3 values) and the element-blocked geometry (7 NE (N+1)^3)
// -- into a two-stage shared-memory ring with cp.async.bulk; while the block
// computes group g the copy of its next group is in flight, so the kernel
// keeps enough bytes moving without needing many resident warps.
#include <stdint.h>

#include "ax_launch.cuh"
#include "tma.cuh"

// Tile shape of the staged kernel: about TH threads per block (whole
// elements of NP^2 threads) and ST ring stages.
template <int NP, int TH, int ST>
struct TmaAxCfg {
    static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    static constexpr int NE = (TH / NP2) > 0 ? TH / NP2 : 1;
    static constexpr int THREADS = NE * NP2;
    static constexpr int STAGES = ST;
    static constexpr size_t U_BYTES = sizeof(float) * NE * NP3;
    static constexpr size_t G_BYTES = sizeof(float) * 7 * NE * NP3;
    static constexpr size_t STAGE_BYTES = U_BYTES + G_BYTES;
    static constexpr size_t WORK_OFF = STAGES * STAGE_BYTES;
    static constexpr size_t WORK_BYTES = sizeof(float) * (2 * NP2 + (size_t)NE * 3 * NP3);
    static constexpr size_t BAR_OFF = (WORK_OFF + WORK_BYTES + 15) / 16 * 16;
    static constexpr size_t SMEM = BAR_OFF + 16 * STAGES;
    // every block copy must be a multiple of 16 bytes
    static constexpr bool OK = (NP3 * sizeof(float)) % 16 == 0 && SMEM <= 227 * 1024;
};

template <int NP, int TH, int ST>
__global__ void __launch_bounds__(TmaAxCfg<NP, TH, ST>::THREADS)
    k_ax_tma(const float *__restrict__ u, float *__restrict__ w, const float *__restrict__ geo,
             const float *__restrict__ D, float h1, float h2, int64_t E, int *err, long long timeout_ns)
{
    using T = TmaAxCfg<NP, TH, ST>;
    using C = T;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + T::BAR_OFF);
    float *work = reinterpret_cast<float *>(smem + T::WORK_OFF);
    float *sD = work, *sDT = work + NP * NP;
    const int grp = threadIdx.x / C::NP2, tid = threadIdx.x - grp * C::NP2;
    float *su = work + 2 * NP * NP + (size_t)grp * 3 * C::NP3;
    float *svr = su + C::NP3, *svs = svr + C::NP3;
    const int64_t groups = (E + C::NE - 1) / C::NE;

    auto issue = [&](int s, int64_t g) {
        const int64_t e0 = g * C::NE;
        const int64_t ne = (E - e0) < C::NE ? (E - e0) : C::NE;
        const uint32_t ub = (uint32_t)(ne * C::NP3 * sizeof(float));
        const uint32_t gb = (uint32_t)(7 * ne * C::NP3 * sizeof(float));
        unsigned char *st = smem + (size_t)s * T::STAGE_BYTES;
        mbar_expect_tx(&bar[s], ub + gb);
        bulk_g2s(st, u + e0 * C::NP3, ub, &bar[s]);
        bulk_g2s(st + T::U_BYTES, geo + e0 * 7 * C::NP3, gb, &bar[s]);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < T::STAGES; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    ax_load_D<NP, float>(D, sD, sDT);
    __syncthreads();
    if (threadIdx.x == 0)
        for (int s = 0; s < T::STAGES; ++s) {
            const int64_t g = blockIdx.x + (int64_t)s * gridDim.x;
            if (g < groups) issue(s, g);
        }
    int64_t it = 0;
    bool failed = false;
    for (;; ++it) {
        const int64_t g = blockIdx.x + it * gridDim.x;
        if (g >= groups) break;
        const int s = (int)(it % T::STAGES);
        const uint32_t parity = (uint32_t)((it / T::STAGES) & 1);
        const bool ok = mbar_wait_bounded(&bar[s], parity, timeout_ns);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const unsigned char *st = smem + (size_t)s * T::STAGE_BYTES;
        const float *su_stage = reinterpret_cast<const float *>(st) + (size_t)grp * C::NP3;
        const float *geo_stage = reinterpret_cast<const float *>(st + T::U_BYTES) + (size_t)grp * 7 * C::NP3;
        const int64_t e = g * C::NE + grp;
        const bool active = grp < C::NE && e < E;
        float *we = w + (active ? e : 0) * C::NP3;
        auto load = [&](int p) { return su_stage[p]; };
        auto store = [&](int p, float v, float) { we[p] = v; };
        ax_element<NP, float>(load, store, geo_stage, h1, h2, sD, sDT, su, svr, svs, tid, active);
        // the stage is free again (ax_element ends with a block barrier)
        if (threadIdx.x == 0) {
            const int64_t g2 = g + (int64_t)T::STAGES * gridDim.x;
            if (g2 < groups) {
                fence_proxy_async_smem();
                issue(s, g2);
            }
        }
    }
    if (failed && threadIdx.x == 0) {
        atomicExch(err, SEM_ERR_TIMEOUT);
        // wait (bounded) for this block's copies still in flight before exiting
        for (int64_t k = it; k < it + T::STAGES; ++k) {
            const int64_t g = blockIdx.x + k * gridDim.x;
            if (g >= groups) break;
            mbar_wait_bounded(&bar[k % T::STAGES], (uint32_t)((k / T::STAGES) & 1), timeout_ns);
        }
    }
}

template <int NP, int TH, int ST>
static int launch_tma(const sem_ctx *c, const float *u, float *w, float h1, float h2, cudaStream_t s)
{
    using T = TmaAxCfg<NP, TH, ST>;
    if constexpr (!T::OK) {
        return SEM_ERR_ARG;
    } else {
        auto kern = k_ax_tma<NP, TH, ST>;
        static std::atomic<unsigned> attr{0};
        SEM_CUDA(sem_smem_attr(kern, T::SMEM, attr));
        int per_sm = 0;
        SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T::THREADS, T::SMEM));
        if (per_sm < 1) return SEM_ERR_ARG;
        const int64_t groups = sem_ceil_div(c->E, T::NE);
        int64_t grid = (int64_t)per_sm * c->num_sms;
        if (grid > groups) grid = groups;
        kern<<<(unsigned)grid, T::THREADS, T::SMEM, s>>>(u, w, c->geo32, c->tab32 + 2 * c->n, h1, h2, c->E,
                                                         (int *)c->err_dev, 2000000000LL);
        SEM_CHECK_LAUNCH();
        return SEM_OK;
    }
}

// Variants of the FP32 operator (see sem_tune_ax): 0 direct loads, 1 staged
// 256 threads x 2 stages, 2 staged 128 threads x 3 stages.
int sem_launch_ax_f32_variant(const sem_ctx *c, int variant, const float *u, float *w, float h1,
                              float h2, cudaStream_t s)
{
    const int n = c->n;
    const bool staged_ok = ((uintptr_t)u % 16) == 0 && c->err_dev && (n == 4 || n == 6 || n == 8 || n == 10);
    if (variant != 0 && staged_ok) {
        switch (n * 8 + variant) {
            case 4 * 8 + 1: return launch_tma<4, 256, 2>(c, u, w, h1, h2, s);
            case 6 * 8 + 1: return launch_tma<6, 256, 2>(c, u, w, h1, h2, s);
            case 8 * 8 + 1: return launch_tma<8, 256, 2>(c, u, w, h1, h2, s);
            case 10 * 8 + 1: return launch_tma<10, 256, 2>(c, u, w, h1, h2, s);
            case 4 * 8 + 2: return launch_tma<4, 128, 3>(c, u, w, h1, h2, s);
            case 6 * 8 + 2: return launch_tma<6, 128, 3>(c, u, w, h1, h2, s);
            case 8 * 8 + 2: return launch_tma<8, 128, 3>(c, u, w, h1, h2, s);
            case 10 * 8 + 2: return launch_tma<10, 128, 3>(c, u, w, h1, h2, s);
            default: break;
        }
    }
    const float *tab = c->tab32 + 2 * n;
    const float *geo = c->geo32;
    SEM_DISPATCH_NP(n, return launch_ax<NP, float>(c, u, w, geo, tab, h1, h2, s));
    return SEM_ERR_ARG;
}
