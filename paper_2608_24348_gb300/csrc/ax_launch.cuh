// ax_launch.cuh -- the stand-alone sem_ax kernel (grid-stride over element
// groups) and its launcher; instantiated per precision in ax_f64.cu / ax_f32.cu.
#pragma once
#include "ax.cuh"
#include "common.cuh"

// ---------------------------------------------------------------------------
// sem_ax: grid-stride over element groups
// ---------------------------------------------------------------------------

template <int NP, typename T>
__global__ void __launch_bounds__(AxCfg<NP>::THREADS)
    k_ax(const T *__restrict__ u, T *__restrict__ w, const T *__restrict__ geo,
         const T *__restrict__ D, T h1, T h2, int64_t E)
{
    using C = AxCfg<NP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *sD = sm, *sDT = sm + NP * NP;
    const int grp = threadIdx.x / C::NP2, tid = threadIdx.x - grp * C::NP2;
    T *su = sm + 2 * NP * NP + (size_t)grp * 3 * C::NP3;
    T *svr = su + C::NP3, *svs = svr + C::NP3;
    ax_load_D<NP, T>(D, sD, sDT);
    for (int64_t e0 = (int64_t)blockIdx.x * C::NE; e0 < E; e0 += (int64_t)gridDim.x * C::NE) {
        const int64_t e = e0 + grp;
        const bool active = e < E;
        const int64_t off = (active ? e : 0) * C::NP3;
        const T *ue = u + off;
        T *we = w + off;
        auto load = [&](int p) { return ue[p]; };
        auto store = [&](int p, T v, T) { we[p] = v; };
        ax_element<NP, T>(load, store, geo + (active ? e : 0) * 7 * C::NP3, h1, h2, sD, sDT, su, svr,
                          svs, tid, active);
    }
}

template <int NP, typename T>
int launch_ax(const sem_ctx *c, const T *u, T *w, const T *geo, const T *D, T h1, T h2,
                     cudaStream_t s)
{
    using C = AxCfg<NP>;
    size_t smem = ax_smem_bytes<NP, T>();
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(k_ax<NP, T>, smem, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax<NP, T>, C::THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t groups = sem_ceil_div(c->E, C::NE);
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > groups) grid = groups;
    if (grid < 1) grid = 1;
    k_ax<NP, T><<<(unsigned)grid, C::THREADS, smem, s>>>(u, w, geo, D, h1, h2, c->E);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

