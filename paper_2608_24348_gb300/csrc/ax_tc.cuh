// ax_tc.cuh -- element operator with 16-bit tensor-core contractions.
//
// The same operator as ax.cuh (Sec. 4, Table 2 rows B-6/B-7: ax_helm with
// fp16 compute), with each of the six directional contractions recast as a
// GEMM of shape (NP^2 x NP) = (NP^2 x NP)(NP x NP):
//     gradient   C_a[m, o] = sum_l A_a[m, l] D[o, l]
//     transpose  W_a[m, o] = sum_l V_a[m, l] D[l, o]
// where the row index m enumerates the two indices not contracted in
// direction a (r: (k,j); s: (k,i); t: (j,i)).  The slab is rounded to BF16 or
// FP16 and multiplied on the tensor cores (mma.sync m16n8k16, FP32
// accumulation); the geometric factors, the h2 B u term and the sum of the
// three transposed contributions stay in FP32.  One warp owns one element;
// its slabs live in a warp-private part of shared memory.  Orders up to
// N = 9 (NP <= 10).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

template <int NP>
struct TcCfg {
    static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    static constexpr int MT = (NP2 + 15) / 16;  // 16-row tiles
    static constexpr int NT = (NP + 7) / 8;     // 8-column tiles
    static constexpr int NE = NP <= 8 ? 8 : 4;  // elements (warps) per 256-thread block
    static constexpr size_t PER_ELEM = (size_t)NP3 * 2 * 4 + (size_t)NP3 * 4 * 3;
    static constexpr bool OK = NP <= 10;
};

template <int NP>
__host__ __device__ constexpr size_t ax_tc_smem_bytes()
{
    return TcCfg<NP>::OK ? TcCfg<NP>::NE * TcCfg<NP>::PER_ELEM : 0;
}

__device__ __forceinline__ uint16_t tc_bits(float x, int fp16)
{
    if (fp16) return __half_as_ushort(__float2half_rn(x));
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ uint32_t tc_pack(uint16_t lo, uint16_t hi)
{
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ void tc_mma(float c[4], const uint32_t a[4], const uint32_t b[2], int fp16)
{
    if (fp16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
}

// Node index of (row m, contracted/output index l) for direction a.
template <int NP>
__device__ __forceinline__ int tc_node(int a, int m, int l)
{
    if (a == 0) return m * NP + l;                            // m = (k, j), l = i
    if (a == 1) return ((m / NP) * NP + l) * NP + (m % NP);   // m = (k, i), l = j
    return l * NP * NP + m;                                   // m = (j, i), l = k
}

// Directional contractions of a 16-bit slab `src` (NP^3) into FP32 `dst`
// (three slabs), with B fragments b[nt][2].
template <int NP>
__device__ __forceinline__ void tc_contract3(const uint16_t *src, int src_stride, float *dst,
                                             const uint32_t b[][2], int lane, int fp16)
{
    using C = TcCfg<NP>;
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint16_t *s = src + a * src_stride;
        float *d = dst + a * C::NP3;
#pragma unroll
        for (int mt = 0; mt < C::MT; ++mt) {
            const int m0 = mt * 16 + gid, m1 = m0 + 8;
            uint32_t af[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = (h & 1) ? m1 : m0;
                const int l = tig * 2 + ((h & 2) ? 8 : 0);
                uint16_t v0 = 0, v1 = 0;
                if (m < C::NP2) {
                    if (l < NP) v0 = s[tc_node<NP>(a, m, l)];
                    if (l + 1 < NP) v1 = s[tc_node<NP>(a, m, l + 1)];
                }
                af[h] = tc_pack(v0, v1);
            }
#pragma unroll
            for (int nt = 0; nt < C::NT; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                tc_mma(c, af, b[nt], fp16);
                const int o0 = nt * 8 + tig * 2;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int m = (h & 2) ? m1 : m0;
                    const int o = o0 + (h & 1);
                    if (m < C::NP2 && o < NP) d[tc_node<NP>(a, m, o)] = c[h];
                }
            }
        }
    }
}

// One element on one warp.  load(q) / store(q, w, u) take global node indices.
template <int NP, class Load, class Store>
__device__ __forceinline__ void ax_tc_element(const Load &load, const Store &store,
                                              const float *__restrict__ geo32,
                                              const float *__restrict__ D32, float h1, float h2,
                                              int64_t e, int fp16, unsigned char *wsm, int lane)
{
    using C = TcCfg<NP>;
    constexpr int PER = (C::NP3 + 31) / 32;
    uint16_t *u16 = reinterpret_cast<uint16_t *>(wsm);
    uint16_t *v16 = u16 + C::NP3;
    float *fb = reinterpret_cast<float *>(v16 + 3 * C::NP3);
    const int gid = lane >> 2, tig = lane & 3;
    const int64_t off = e * C::NP3;
    float ureg[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int q = lane + 32 * t;
        if (q < C::NP3) {
            const float x = load(off + q);
            ureg[t] = x;
            u16[q] = tc_bits(x, fp16);
        }
    }
    // B fragments: gradient uses B[l][o] = D[o][l], transpose B[l][o] = D[l][o]
    uint32_t bT[C::NT][2], bN[C::NT][2];
#pragma unroll
    for (int nt = 0; nt < C::NT; ++nt) {
        const int o = nt * 8 + gid;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = tig * 2 + 8 * h;
            float t0 = 0.f, t1 = 0.f, n0 = 0.f, n1 = 0.f;
            if (o < NP && l < NP) { t0 = D32[o * NP + l]; n0 = D32[l * NP + o]; }
            if (o < NP && l + 1 < NP) { t1 = D32[o * NP + l + 1]; n1 = D32[(l + 1) * NP + o]; }
            bT[nt][h] = tc_pack(tc_bits(t0, fp16), tc_bits(t1, fp16));
            bN[nt][h] = tc_pack(tc_bits(n0, fp16), tc_bits(n1, fp16));
        }
    }
    __syncwarp();
    tc_contract3<NP>(u16, 0, fb, bT, lane, fp16);
    __syncwarp();
    const float *G = geo32 + e * 7 * C::NP3;
    float wacc[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int q = lane + 32 * t;
        if (q < C::NP3) {
            const float ur = fb[q], us = fb[C::NP3 + q], ut = fb[2 * C::NP3 + q];
            const float g11 = G[0 * C::NP3 + q], g22 = G[1 * C::NP3 + q], g33 = G[2 * C::NP3 + q];
            const float g12 = G[3 * C::NP3 + q], g13 = G[4 * C::NP3 + q], g23 = G[5 * C::NP3 + q];
            const float bm = G[6 * C::NP3 + q];
            v16[q] = tc_bits(h1 * (g11 * ur + g12 * us + g13 * ut), fp16);
            v16[C::NP3 + q] = tc_bits(h1 * (g12 * ur + g22 * us + g23 * ut), fp16);
            v16[2 * C::NP3 + q] = tc_bits(h1 * (g13 * ur + g23 * us + g33 * ut), fp16);
            wacc[t] = h2 * bm * ureg[t];
        }
    }
    __syncwarp();
    tc_contract3<NP>(v16, C::NP3, fb, bN, lane, fp16);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int q = lane + 32 * t;
        if (q < C::NP3) store(off + q, wacc[t] + fb[q] + fb[C::NP3 + q] + fb[2 * C::NP3 + q], ureg[t]);
    }
    __syncwarp();
}

// A group of NE elements on a 256-thread block (one element per warp).
template <int NP, class Load, class Store>
__device__ __forceinline__ void ax_tc_group(const Load &load, const Store &store,
                                            const float *__restrict__ geo32,
                                            const float *__restrict__ D32, float h1, float h2,
                                            int64_t E, int64_t g, int fp16, unsigned char *smem)
{
    if constexpr (TcCfg<NP>::OK) {
        using C = TcCfg<NP>;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t e = g * C::NE + warp;
        if (warp < C::NE && e < E)
            ax_tc_element<NP>(load, store, geo32, D32, h1, h2, e, fp16,
                              smem + (size_t)warp * C::PER_ELEM, lane);
    }
}
