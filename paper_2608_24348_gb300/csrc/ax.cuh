// ax.cuh -- the matrix-free element operator on CUDA cores (FP64 / FP32).
//
// ax_helm (Sec. 4, Table 2 rows B-6/B-7) on one hexahedral element of order
// N = NP - 1:
//     u_a = D_a u                     (a = r, s, t; D_r = I x I x D, ...)
//     v_a = h1 sum_b G_ab u_b         (six symmetric geometric factors)
//     w   = sum_a D_a^T v_a + h2 B u
//
// Thread layout: NP*NP threads per element, thread (i, j) owns the column
// u[0..NP-1][j][i] in registers.  The t-direction contractions stay in
// registers; the r and s contractions read the element slab in shared memory.
// D is kept twice in shared memory (D and D^T) so that every read is either a
// broadcast or unit-stride across a warp.  Geometric factors are streamed
// once from HBM, coalesced (element-blocked [7][NP^3] layout).
#pragma once

template <int NP>
struct AxCfg {
    static constexpr int NP2 = NP * NP;
    static constexpr int NP3 = NP2 * NP;
    // elements per 256-thread block
    static constexpr int NE = (256 / NP2) > 0 ? (256 / NP2) : 1;
    static constexpr int THREADS = NE * NP2;
};

// Shared memory: sD[NP*NP], sDT[NP*NP], then per element u, vr, vs slabs.
template <int NP, typename T>
__host__ __device__ constexpr size_t ax_smem_bytes()
{
    return sizeof(T) * (2 * NP * NP + (size_t)AxCfg<NP>::NE * 3 * NP * NP * NP);
}

template <int NP, typename T>
__device__ __forceinline__ void ax_load_D(const T *__restrict__ D, T *sD, T *sDT)
{
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) {
        int a = t / NP, b = t - a * NP;
        T v = D[t];
        sD[t] = v;            // sD[a*NP + b]  = D_ab
        sDT[b * NP + a] = v;  // sDT[b*NP + a] = D_ab
    }
}

// One element.  All threads of the block must call it (it synchronises);
// `active` is false for threads without an element.  load(p) returns u at
// local node p; store(p, w, u) receives w and the input value at node p.
template <int NP, typename T, class Load, class Store>
__device__ __forceinline__ void ax_element(const Load &load, const Store &store,
                                           const T *__restrict__ geo, T h1, T h2,
                                           const T *__restrict__ sD, const T *__restrict__ sDT,
                                           T *__restrict__ su, T *__restrict__ svr,
                                           T *__restrict__ svs, int tid, bool active)
{
    constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    const int i = tid % NP, j = tid / NP;
    T ru[NP], rvt[NP], rw[NP];
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            ru[k] = load(k * NP2 + tid);
            su[k * NP2 + tid] = ru[k];
        }
    }
    __syncthreads();  // publishes the slab and the D tables written before the call
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                ur = fma(sDT[l * NP + i], su[k * NP2 + j * NP + l], ur);
                us = fma(sDT[l * NP + j], su[k * NP2 + l * NP + i], us);
                ut = fma(sDT[l * NP + k], ru[l], ut);
            }
            const int p = k * NP2 + tid;
            const T g11 = geo[0 * NP3 + p], g22 = geo[1 * NP3 + p], g33 = geo[2 * NP3 + p];
            const T g12 = geo[3 * NP3 + p], g13 = geo[4 * NP3 + p], g23 = geo[5 * NP3 + p];
            const T bm = geo[6 * NP3 + p];
            svr[p] = h1 * (g11 * ur + g12 * us + g13 * ut);
            svs[p] = h1 * (g12 * ur + g22 * us + g23 * ut);
            rvt[k] = h1 * (g13 * ur + g23 * us + g33 * ut);
            rw[k] = h2 * bm * ru[k];
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            T s = rw[k];
#pragma unroll
            for (int l = 0; l < NP; ++l) {
                s = fma(sD[l * NP + i], svr[k * NP2 + j * NP + l], s);
                s = fma(sD[l * NP + j], svs[k * NP2 + l * NP + i], s);
                s = fma(sD[l * NP + k], rvt[l], s);
            }
            store(k * NP2 + tid, s, ru[k]);
        }
    }
    __syncthreads();
}

// Low-register variant: one thread per node (strided over the element),
// every contraction read from shared memory.  Used where register pressure
// matters more than speed (the FP64 residual of mixed-precision refinement,
// evaluated once per refinement step).  smem: u, vr, vs, vt slabs.
template <int NP>
__host__ __device__ constexpr size_t ax_lowreg_smem_bytes()
{
    return sizeof(double) * (2 * NP * NP + 4 * (size_t)NP * NP * NP);
}

template <int NP, class Load, class Store>
__device__ __forceinline__ void ax_element_lowreg(const Load &load, const Store &store,
                                                  const double *__restrict__ geo, double h1,
                                                  double h2, const double *__restrict__ D,
                                                  unsigned char *smem, bool active)
{
    constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    double *sD = reinterpret_cast<double *>(smem), *sDT = sD + NP2;
    double *su = sDT + NP2, *svr = su + NP3, *svs = svr + NP3, *svt = svs + NP3;
    for (int t = threadIdx.x; t < NP2; t += blockDim.x) {
        const int a = t / NP, b = t - a * NP;
        sD[t] = D[t];
        sDT[b * NP + a] = D[t];
    }
    if (active)
        for (int q = threadIdx.x; q < NP3; q += blockDim.x) su[q] = load(q);
    __syncthreads();
    if (active)
        for (int q = threadIdx.x; q < NP3; q += blockDim.x) {
            const int i = q % NP, j = (q / NP) % NP, k = q / NP2;
            double ur = 0, us = 0, ut = 0;
            for (int l = 0; l < NP; ++l) {
                ur = fma(sDT[l * NP + i], su[(k * NP + j) * NP + l], ur);
                us = fma(sDT[l * NP + j], su[(k * NP + l) * NP + i], us);
                ut = fma(sDT[l * NP + k], su[(l * NP + j) * NP + i], ut);
            }
            const double g11 = geo[0 * NP3 + q], g22 = geo[1 * NP3 + q], g33 = geo[2 * NP3 + q];
            const double g12 = geo[3 * NP3 + q], g13 = geo[4 * NP3 + q], g23 = geo[5 * NP3 + q];
            svr[q] = h1 * (g11 * ur + g12 * us + g13 * ut);
            svs[q] = h1 * (g12 * ur + g22 * us + g23 * ut);
            svt[q] = h1 * (g13 * ur + g23 * us + g33 * ut);
        }
    __syncthreads();
    if (active)
        for (int q = threadIdx.x; q < NP3; q += blockDim.x) {
            const int i = q % NP, j = (q / NP) % NP, k = q / NP2;
            double s = h2 * geo[6 * NP3 + q] * su[q];
            for (int l = 0; l < NP; ++l) {
                s = fma(sD[l * NP + i], svr[(k * NP + j) * NP + l], s);
                s = fma(sD[l * NP + j], svs[(k * NP + l) * NP + i], s);
                s = fma(sD[l * NP + k], svt[(l * NP + j) * NP + i], s);
            }
            store(q, s, su[q]);
        }
    __syncthreads();
}
