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

// ---------------------------------------------------------------------------
// Split-operand contractions (FP32-level accuracy from 16-bit tensor cores)
// ---------------------------------------------------------------------------
// Every contracted value x is split into 16-bit parts, x = x1 + x2 (FP16, 11
// significant bits each) or x = x1 + x2 + x3 (BF16, 8 bits each), and so is
// D.  The products that carry about 2^-22 relative accuracy are summed by the
// tensor cores with FP32 accumulation; two parts stacked along K fill the
// 16-wide K of one m16n8k16 MMA when N+1 <= 8:
//   FP16 x2:  [x1|x2][D1;D1] + [x1|x2][D2;0]           (dropped: x2 D2)
//   BF16 x3:  [x1|x2][D1;D1] + [x1|x2][D2;D2] + [x3|x1][D1;D3]
//             (dropped: x2 D3, x3 D2, x3 D3, all of order 2^-24).
// FP16 parts need their magnitude inside FP16's range: each element's input
// and each directional flux is scaled by a power of two first (exact), and
// the result scaled back.  BF16 has FP32's exponent range.
template <int NP>
struct TcSplitCfg {
    static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    static constexpr int MT = (NP2 + 15) / 16;
    static constexpr int NE = 8;  // one element per warp, 256-thread blocks
    // gradient slabs (3 NP^3 floats), output accumulator (NP^3 floats), three 16-bit parts
    static constexpr size_t PER_ELEM = (size_t)NP3 * 4 * 4 + (size_t)NP3 * 2 * 3;
    static constexpr bool OK = NP <= 8;
};

template <int NP>
__host__ __device__ constexpr size_t ax_tc_split_smem_bytes()
{
    return TcSplitCfg<NP>::OK ? TcSplitCfg<NP>::NE * TcSplitCfg<NP>::PER_ELEM : 0;
}

// x = p1 + p2 (+ p3) in 16-bit parts, each the rounding of what remains.
template <bool FP16>
__device__ __forceinline__ void tc_split(float x, uint16_t &p1, uint16_t &p2, uint16_t &p3)
{
    if constexpr (FP16) {
        const __half a = __float2half_rn(x);
        p1 = __half_as_ushort(a);
        p2 = __half_as_ushort(__float2half_rn(x - __half2float(a)));
        p3 = 0;
    } else {
        const __nv_bfloat16 a = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(a);
        const __nv_bfloat16 b = __float2bfloat16_rn(r1);
        p1 = __bfloat16_as_ushort(a);
        p2 = __bfloat16_as_ushort(b);
        p3 = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(b)));
    }
}

// 2^-(e+1) for the exponent e of m (m >= 0 finite), as a float: |x| <= m
// gives |x * scale| < 1.  Zero m gives 1.
__device__ __forceinline__ float tc_unit_scale(float m)
{
    const int e = (int)((__float_as_uint(m) >> 23) & 0xff);  // biased exponent of m
    if (e == 0) return 1.0f;
    int se = 127 - (e - 127 + 1);
    se = se < 1 ? 1 : (se > 254 ? 254 : se);
    return __uint_as_float((unsigned)se << 23);
}

// One direction's contraction of the split parts (P[k] arrays of NP^3 16-bit
// values) into FP32 c, which the caller stores (or adds) at node
// tc_node(a, m, o).  BFR[t] are the B fragments of the MMAs.
template <int NP, bool FP16, class Out>
__device__ __forceinline__ void tc_contract_split(int a, const uint16_t *const P[3], const uint32_t bfr[3][2],
                                                  int lane, const Out &out)
{
    using C = TcSplitCfg<NP>;
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mt = 0; mt < C::MT; ++mt) {
        const int m0 = mt * 16 + gid, m1 = m0 + 8;
        // A fragments: [part 0 | part 1] and (BF16) [part 2 | part 0]
        uint32_t A01[4], A20[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int m = (h & 1) ? m1 : m0;
            const int l = tig * 2;
            const bool hi = (h & 2) != 0;
            uint16_t x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            if (m < C::NP2) {
                const uint16_t *pa = hi ? P[1] : P[0];
                if (l < NP) x0 = pa[tc_node<NP>(a, m, l)];
                if (l + 1 < NP) x1 = pa[tc_node<NP>(a, m, l + 1)];
                if constexpr (!FP16) {
                    const uint16_t *pb = hi ? P[0] : P[2];
                    if (l < NP) y0 = pb[tc_node<NP>(a, m, l)];
                    if (l + 1 < NP) y1 = pb[tc_node<NP>(a, m, l + 1)];
                }
            }
            A01[h] = tc_pack(x0, x1);
            A20[h] = tc_pack(y0, y1);
        }
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tc_mma(c, A01, bfr[0], FP16 ? 1 : 0);
        tc_mma(c, A01, bfr[1], FP16 ? 1 : 0);
        if constexpr (!FP16) tc_mma(c, A20, bfr[2], 0);
        const int o0 = tig * 2;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int m = (h & 2) ? m1 : m0;
            const int o = o0 + (h & 1);
            if (m < C::NP2 && o < NP) out(tc_node<NP>(a, m, o), c[h]);
        }
    }
}

// One element on one warp with split-operand contractions (N+1 <= 8).
// load(q) / store(q, w, u) take global node indices.
template <int NP, bool FP16, class Load, class Store>
__device__ __forceinline__ void ax_tc_split_element(const Load &load, const Store &store,
                                                    const float *__restrict__ geo32,
                                                    const float *__restrict__ D32, float h1, float h2,
                                                    int64_t e, unsigned char *wsm, int lane)
{
    using C = TcSplitCfg<NP>;
    constexpr int PER = (C::NP3 + 31) / 32;
    float *fb = reinterpret_cast<float *>(wsm);          // 3 NP^3: gradient
    float *acc = fb + 3 * C::NP3;                         // NP^3: transposed sum
    uint16_t *P0 = reinterpret_cast<uint16_t *>(acc + C::NP3);
    uint16_t *P1 = P0 + C::NP3, *P2 = P1 + C::NP3;
    const uint16_t *const P[3] = {P0, P1, P2};
    const int64_t off = e * C::NP3;
    const int gid = lane >> 2, tig = lane & 3;
    // D in parts, as B fragments: gradient B[l][o] = D[o][l], transpose B[l][o] = D[l][o]
    uint32_t bG[3][2], bT[3][2];
    {
        const int o = gid, l = tig * 2;
        float dg[2][2], dt[2][2];  // [row pair][element]
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            dg[r][0] = dg[r][1] = dt[r][0] = dt[r][1] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int ll = l + k;
            if (o < NP && ll < NP) {
                dg[0][k] = D32[o * NP + ll];
                dt[0][k] = D32[ll * NP + o];
            }
        }
        uint16_t g1[2], g2[2], g3[2], t1[2], t2[2], t3[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            tc_split<FP16>(dg[0][k], g1[k], g2[k], g3[k]);
            tc_split<FP16>(dt[0][k], t1[k], t2[k], t3[k]);
        }
        // MMA 0: [x1|x2][D1;D1]; MMA 1: FP16 [x1|x2][D2;0], BF16 [x1|x2][D2;D2]; MMA 2 (BF16): [x3|x1][D1;D3]
        bG[0][0] = tc_pack(g1[0], g1[1]); bG[0][1] = tc_pack(g1[0], g1[1]);
        bT[0][0] = tc_pack(t1[0], t1[1]); bT[0][1] = tc_pack(t1[0], t1[1]);
        bG[1][0] = tc_pack(g2[0], g2[1]); bG[1][1] = FP16 ? 0u : tc_pack(g2[0], g2[1]);
        bT[1][0] = tc_pack(t2[0], t2[1]); bT[1][1] = FP16 ? 0u : tc_pack(t2[0], t2[1]);
        bG[2][0] = tc_pack(g1[0], g1[1]); bG[2][1] = tc_pack(g3[0], g3[1]);
        bT[2][0] = tc_pack(t1[0], t1[1]); bT[2][1] = tc_pack(t3[0], t3[1]);
    }
    // input, its scale, parts
    float ureg[PER];
    float mu = 0.f;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int q = lane + 32 * t;
        ureg[t] = q < C::NP3 ? load(off + q) : 0.f;
        mu = fmaxf(mu, fabsf(ureg[t]));
    }
    float su = 1.f;
    if constexpr (FP16) su = tc_unit_scale(__uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mu))));
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int q = lane + 32 * t;
        if (q < C::NP3) {
            uint16_t a, b, c;
            tc_split<FP16>(ureg[t] * su, a, b, c);
            P0[q] = a;
            P1[q] = b;
            P2[q] = c;
        }
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 3; ++a)
        tc_contract_split<NP, FP16>(a, P, bG, lane, [&](int node, float v) { fb[a * C::NP3 + node] = v; });
    __syncwarp();
    const float *G = geo32 + e * 7 * C::NP3;
    // one direction of fluxes at a time: v_a = h1 sum_b G_ab g_b, split, contracted with D^T
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float vreg[PER];
        float mv = 0.f;
        const int c0 = a == 0 ? 0 : (a == 1 ? 3 : 4), c1 = a == 0 ? 3 : (a == 1 ? 1 : 5),
                  c2 = a == 0 ? 4 : (a == 1 ? 5 : 2);
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int q = lane + 32 * t;
            vreg[t] = 0.f;
            if (q < C::NP3) {
                const float ur = fb[q], us = fb[C::NP3 + q], ut = fb[2 * C::NP3 + q];
                vreg[t] = h1 * (G[c0 * C::NP3 + q] * ur + G[c1 * C::NP3 + q] * us + G[c2 * C::NP3 + q] * ut);
                mv = fmaxf(mv, fabsf(vreg[t]));
            }
        }
        float sv = 1.f;
        if constexpr (FP16) sv = tc_unit_scale(__uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mv))));
        __syncwarp();  // the previous direction's contraction has read the parts
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int q = lane + 32 * t;
            if (q < C::NP3) {
                uint16_t x, y, z;
                tc_split<FP16>(vreg[t] * sv, x, y, z);
                P0[q] = x;
                P1[q] = y;
                P2[q] = z;
            }
        }
        __syncwarp();
        // undo both scales (powers of two: exact unless the result leaves FP32's range)
        const float bu = 1.0f / su, bv = 1.0f / sv;
        if (a == 0)
            tc_contract_split<NP, FP16>(a, P, bT, lane, [&](int node, float v) { acc[node] = (v * bv) * bu; });
        else
            tc_contract_split<NP, FP16>(a, P, bT, lane, [&](int node, float v) { acc[node] += (v * bv) * bu; });
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int q = lane + 32 * t;
        if (q < C::NP3) store(off + q, h2 * G[6 * C::NP3 + q] * ureg[t] + acc[q], ureg[t]);
    }
    __syncwarp();
}

// A group of 8 elements on a 256-thread block (one element per warp).
template <int NP, bool FP16, class Load, class Store>
__device__ __forceinline__ void ax_tc_split_group(const Load &load, const Store &store,
                                                  const float *__restrict__ geo32,
                                                  const float *__restrict__ D32, float h1, float h2,
                                                  int64_t E, int64_t g, unsigned char *smem)
{
    if constexpr (TcSplitCfg<NP>::OK) {
        using C = TcSplitCfg<NP>;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t e = g * C::NE + warp;
        if (warp < C::NE && e < E)
            ax_tc_split_element<NP, FP16>(load, store, geo32, D32, h1, h2, e,
                                          smem + (size_t)warp * C::PER_ELEM, lane);
    }
}
