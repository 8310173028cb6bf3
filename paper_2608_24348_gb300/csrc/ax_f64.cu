// ax_f64.cu -- F64 instantiations of the stand-alone element operator: the
// folded (even-odd) kernel for even N+1, the unfolded one otherwise.
#include "ax_eo64.cuh"
#include "ax_launch.cuh"

// The four half tables, by value (constant bank), copied to shared memory.
struct Eo64Tabs {
    double t[4 * (SEM_NPMAX / 2) * (SEM_NPMAX / 2)];
};

template <int NP>
__global__ void __launch_bounds__(AxEo64Cfg<NP>::THREADS)
    k_ax_eo64(const double *__restrict__ u, double *__restrict__ w, const double *__restrict__ geo,
              const __grid_constant__ Eo64Tabs tabs, double h1, double h2, int64_t E)
{
    using C = AxEo64Cfg<NP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sm = reinterpret_cast<double *>(smem_raw);
    double *stab = sm;
    const int grp = threadIdx.x / C::NP2, tid = threadIdx.x - grp * C::NP2;
    double *slab = sm + 4 * C::H * C::H + (size_t)grp * 5 * C::SLAB;
    for (int t = threadIdx.x; t < 4 * C::H * C::H; t += blockDim.x) stab[t] = tabs.t[t];
    // (published by the element's first barrier)
    for (int64_t e0 = (int64_t)blockIdx.x * C::NE; e0 < E; e0 += (int64_t)gridDim.x * C::NE) {
        const int64_t e = e0 + grp;
        const bool active = e < E;
        const int64_t off = (active ? e : 0) * C::NP3;
        const double *ue = u + off;
        double *we = w + off;
        auto load = [&](int p) { return ue[p]; };
        auto store = [&](int p, double v, double) { we[p] = v; };
        ax_eo64_element<NP>(load, store, geo + (active ? e : 0) * 7 * C::NP3, h1, h2, stab, slab, tid, active);
    }
}

template <int NP>
static int launch_ax_eo64(const sem_ctx *c, const double *u, double *w, double h1, double h2, cudaStream_t s)
{
    using C = AxEo64Cfg<NP>;
    Eo64Tabs tabs;
    memset(&tabs, 0, sizeof(tabs));
    ax_eo64_tables(NP, c->hD, tabs.t);
    const size_t smem = ax_eo64_smem_bytes<NP>();
    static std::atomic<unsigned> attr{0};
    SEM_CUDA(sem_smem_attr(k_ax_eo64<NP>, smem, attr));
    int per_sm = 0;
    SEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ax_eo64<NP>, C::THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t groups = sem_ceil_div(c->E, C::NE);
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > groups) grid = groups;
    if (grid < 1) grid = 1;
    k_ax_eo64<NP><<<(unsigned)grid, C::THREADS, smem, s>>>(u, w, c->geo64, tabs, h1, h2, c->E);
    SEM_CHECK_LAUNCH();
    return SEM_OK;
}

// fold = 0 forces the unfolded kernel (the tuner's other candidate).
int sem_launch_ax_f64_v(const sem_ctx *c, const double *u, double *w, double h1, double h2, int fold,
                        cudaStream_t s)
{
    const int n = c->n;
    const double *tab = c->tab64 + 2 * n;
    const double *geo = c->geo64;
    if (fold && n % 2 == 0) {
        switch (n) {
            case 2: return launch_ax_eo64<2>(c, u, w, h1, h2, s);
            case 4: return launch_ax_eo64<4>(c, u, w, h1, h2, s);
            case 6: return launch_ax_eo64<6>(c, u, w, h1, h2, s);
            case 8: return launch_ax_eo64<8>(c, u, w, h1, h2, s);
            case 10: return launch_ax_eo64<10>(c, u, w, h1, h2, s);
            case 12: return launch_ax_eo64<12>(c, u, w, h1, h2, s);
            case 14: return launch_ax_eo64<14>(c, u, w, h1, h2, s);
            case 16: return launch_ax_eo64<16>(c, u, w, h1, h2, s);
            default: break;
        }
    }
    SEM_DISPATCH_NP(n, return launch_ax<NP, double>(c, u, w, geo, tab, h1, h2, s));
    return SEM_ERR_ARG;
}

int sem_launch_ax_f64(const sem_ctx *c, const double *u, double *w, double h1, double h2, cudaStream_t s)
{
    return sem_launch_ax_f64_v(c, u, w, h1, h2, 1, s);
}
