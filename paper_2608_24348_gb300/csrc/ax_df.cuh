// ax_df.cuh -- FP64-accurate element operator evaluated on the FP32 pipes.
//
// GB300 executes FP64 FMAs at 1/58 of its FP32 rate, which makes the plain FP64
// operator ALU-bound far below the HBM roofline.  This variant keeps FP64
// inputs and outputs and FP64-level accuracy but does its arithmetic in pairs
// of FP32 numbers (a "double-float" hi + lo with |lo| <= ulp(hi)/2):
//   - products are made exact with TwoProd (Dekker 1971, via FMA),
//   - sums use TwoSum (Knuth 1969) for the leading part and collect all
//     rounding errors in a second accumulator, which is the compensated dot
//     product Dot2 of Ogita, Rump & Oishi (2005): the result is as accurate as
//     if computed in twice the working precision (about 2^-48) and rounded,
//   - before splitting, every element's input is scaled by a power of two
//     (exact) so that its largest entry is of order one; the output is scaled
//     back, so the FP32 exponent range never limits an FP64 input.
// The geometric factors and D are stored as float pairs (same bytes as FP64).
// The three intrinsics-only helpers below are never contracted or reassociated
// by the compiler (__fmul_rn / __fadd_rn / __fsub_rn / __fmaf_rn).
#pragma once

#include <stdint.h>

struct dfp {
    float hi, lo;
};

// Compensated accumulator: s is the running sum, e gathers the rounding errors.
struct dfacc {
    float s, e;
};

// Biased exponent field of a double (0 for zero and subnormals).
__device__ __forceinline__ int df_bexp(double x)
{
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// x * 2^-E as a float pair, by integer operations on the bit pattern: hi takes
// the leading 24 significand bits, lo the remaining 29 (rounded to 24).  Parts
// below the FP32 normal range of the scaled element are dropped (they are
// smaller than 2^-74 relative to the element's largest entry).
__device__ __forceinline__ dfp df_split_scaled(double x, int E)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((b >> 52) & 0x7ff);
    const int e = be - 1023 - E;  // scaled value = 1.m x 2^e
    if (be == 0 || e < -126) return {0.f, 0.f};
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((unsigned)(M >> 29) & 0x7fffffu));
    float lo = 0.f;
    if (e >= -74) {
        lo = __uint2float_rn((unsigned)(M & 0x1FFFFFFFull)) * __uint_as_float((unsigned)(e - 52 + 127) << 23);
        lo = __uint_as_float(__float_as_uint(lo) | sign);
    }
    return {hi, lo};
}

// Exact FP32 -> FP64 widening of a normal float (zero and subnormals -> 0).
__device__ __forceinline__ double df_widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xff;
    if (ex == 0) return 0.0;
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                                 ((unsigned long long)(ex - 127 + 1023) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// (hi + lo) * 2^E in FP64: one FP64 addition, the scaling on the exponent field.
__device__ __forceinline__ double df_join_scaled(dfp a, int E)
{
    const double r = df_widen(a.hi) + df_widen(a.lo);
    long long b = __double_as_longlong(r);
    const int be = (int)((b >> 52) & 0x7ff);
    if (be == 0) return 0.0;
    const int nb = be + E;
    if (nb <= 0) return 0.0;
    if (nb >= 0x7ff) return __longlong_as_double((b & (1ll << 63)) | (0x7ffll << 52));
    return __longlong_as_double(b + ((long long)E << 52));
}

// A = a * b: a fresh accumulator holding one exact product (TwoProd) plus the
// cross terms; the same value df_mad would give from a zero accumulator, eight
// operations cheaper.
__device__ __forceinline__ dfacc df_mul(dfp a, dfp b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float err = __fmaf_rn(a.hi, b.hi, -p);
    err = __fmaf_rn(a.hi, b.lo, err);
    err = __fmaf_rn(a.lo, b.hi, err);
    return {p, err};
}

// A += a * b   (a, b float pairs)
__device__ __forceinline__ void df_mad(dfacc &A, dfp a, dfp b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float err = __fmaf_rn(a.hi, b.hi, -p);     // exact low part of a.hi * b.hi
    err = __fmaf_rn(a.hi, b.lo, err);
    err = __fmaf_rn(a.lo, b.hi, err);
    const float s = __fadd_rn(A.s, p);        // TwoSum(A.s, p)
    const float bv = __fsub_rn(s, A.s);
    const float t = __fadd_rn(__fsub_rn(A.s, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    A.s = s;
    A.e = __fadd_rn(A.e, __fadd_rn(t, err));
}

// A += a   (a float pair)
__device__ __forceinline__ void df_add(dfacc &A, dfp a)
{
    const float s = __fadd_rn(A.s, a.hi);
    const float bv = __fsub_rn(s, A.s);
    const float t = __fadd_rn(__fsub_rn(A.s, __fsub_rn(s, bv)), __fsub_rn(a.hi, bv));
    A.s = s;
    A.e = __fadd_rn(A.e, __fadd_rn(t, a.lo));
}

// a + b as a pair that is not renormalised: TwoSum of the leading parts, both
// trailing parts added to the error term (8 operations).  Every consumer of a
// pair (df_mad, df_add, TwoSum, the final FP64 join) is exact or error-bounded
// for such pairs, so renormalising between stages buys no accuracy.
__device__ __forceinline__ dfp df_sum(dfp a, dfp b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    return {s, __fadd_rn(t, __fadd_rn(a.lo, b.lo))};
}

// The accumulator as a pair, without renormalising.
__device__ __forceinline__ dfp df_raw(dfacc A) { return {A.s, A.e}; }

template <int NP>
struct AxDfCfg {
    static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    static constexpr int NE = (256 / NP2) > 0 ? (256 / NP2) : 1;
    static constexpr int THREADS = NE * NP2;
};

// sD, sDT: float pairs of D and D^T; per element three pair slabs + an exponent.
template <int NP>
__host__ __device__ constexpr size_t ax_df_smem_bytes()
{
    return sizeof(dfp) * (2 * NP * NP + (size_t)AxDfCfg<NP>::NE * 3 * NP * NP * NP) +
           sizeof(int) * AxDfCfg<NP>::NE;
}

template <int NP>
__device__ __forceinline__ void ax_df_load_D(const dfp *__restrict__ D, dfp *sD, dfp *sDT)
{
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) {
        const int a = t / NP, b = t - a * NP;
        const dfp v = D[t];
        sD[t] = v;
        sDT[b * NP + a] = v;
    }
}

// One element on NP*NP threads (thread (i, j) owns column u[.][j][i]).
// load(p) -> double, store(p, double w).  All threads of the block call it.
template <int NP, class Load, class Store>
__device__ __forceinline__ void ax_df_element(const Load &load, const Store &store,
                                              const dfp *__restrict__ geo, dfp h1, dfp h2,
                                              const dfp *__restrict__ sD, const dfp *__restrict__ sDT,
                                              dfp *__restrict__ su, dfp *__restrict__ svr,
                                              dfp *__restrict__ svs, int *sexp, int tid, bool active)
{
    constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    const int i = tid % NP, j = tid / NP;
    double xu[NP];
    if (tid == 0) *sexp = 0;
    __syncthreads();
    if (active) {
        int m = 0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            xu[k] = load(k * NP2 + tid);
            m = max(m, df_bexp(xu[k]));
        }
        atomicMax(sexp, m);
    }
    __syncthreads();
    const int E = *sexp > 0 ? *sexp - 1023 : 0;  // element scale 2^E (exact)
    dfp ru[NP], rvt[NP], rw[NP];
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            ru[k] = df_split_scaled(xu[k], E);
            su[k * NP2 + tid] = ru[k];
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            dfacc ar = df_mul(sDT[i], su[k * NP2 + j * NP]);
            dfacc as = df_mul(sDT[j], su[k * NP2 + i]);
            dfacc at = df_mul(sDT[k], ru[0]);
#pragma unroll
            for (int l = 1; l < NP; ++l) {
                df_mad(ar, sDT[l * NP + i], su[k * NP2 + j * NP + l]);
                df_mad(as, sDT[l * NP + j], su[k * NP2 + l * NP + i]);
                df_mad(at, sDT[l * NP + k], ru[l]);
            }
            const dfp ur = df_raw(ar), us = df_raw(as), ut = df_raw(at);
            const int p = k * NP2 + tid;
            const dfp g11 = geo[0 * NP3 + p], g22 = geo[1 * NP3 + p], g33 = geo[2 * NP3 + p];
            const dfp g12 = geo[3 * NP3 + p], g13 = geo[4 * NP3 + p], g23 = geo[5 * NP3 + p];
            const dfp bm = geo[6 * NP3 + p];
            dfacc vr = df_mul(g11, ur), vs = df_mul(g12, ur), vt = df_mul(g13, ur);
            df_mad(vr, g12, us); df_mad(vr, g13, ut);
            df_mad(vs, g22, us); df_mad(vs, g23, ut);
            df_mad(vt, g23, us); df_mad(vt, g33, ut);
            const dfacc vw = df_mul(bm, ru[k]);
            svr[p] = df_raw(vr);
            svs[p] = df_raw(vs);
            rvt[k] = df_raw(vt);
            rw[k] = df_raw(vw);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            dfacc ar = df_mul(sD[i], svr[k * NP2 + j * NP]);  // three independent chains
            dfacc as = df_mul(sD[j], svs[k * NP2 + i]);
            dfacc at = df_mul(sD[k], rvt[0]);
#pragma unroll
            for (int l = 1; l < NP; ++l) {
                df_mad(ar, sD[l * NP + i], svr[k * NP2 + j * NP + l]);
                df_mad(as, sD[l * NP + j], svs[k * NP2 + l * NP + i]);
                df_mad(at, sD[l * NP + k], rvt[l]);
            }
            df_add(ar, df_raw(as));
            df_add(ar, df_raw(at));
            dfacc o = df_mul(h1, df_raw(ar));
            df_mad(o, h2, rw[k]);
            store(k * NP2 + tid, df_join_scaled(df_raw(o), E));
        }
    }
    __syncthreads();
}

// Low-register variant (one thread per node, strided; every contraction read
// from shared memory): the FP64-accurate residual inside mixed-precision
// refinement, where the kernel's register budget belongs to the FP32 phases.
template <int NP>
__host__ __device__ constexpr size_t ax_df_lowreg_smem_bytes()
{
    return sizeof(dfp) * (2 * NP * NP + 4 * (size_t)NP * NP * NP) + 16;
}

template <int NP, class Load, class Store>
__device__ __forceinline__ void ax_df_element_lowreg(const Load &load, const Store &store,
                                                     const dfp *__restrict__ geo, dfp h1, dfp h2,
                                                     const dfp *__restrict__ D, unsigned char *smem)
{
    constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    dfp *sD = reinterpret_cast<dfp *>(smem), *sDT = sD + NP2;
    dfp *su = sDT + NP2, *svr = su + NP3, *svs = svr + NP3, *svt = svs + NP3;
    int *sexp = reinterpret_cast<int *>(svt + NP3);
    for (int t = threadIdx.x; t < NP2; t += blockDim.x) {
        const int a = t / NP, b = t - a * NP;
        sD[t] = D[t];
        sDT[b * NP + a] = D[t];
    }
    if (threadIdx.x == 0) *sexp = 0;
    __syncthreads();
    int m = 0;
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) m = max(m, df_bexp(load(q)));
    atomicMax(sexp, m);
    __syncthreads();
    const int E = *sexp > 0 ? *sexp - 1023 : 0;
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) su[q] = df_split_scaled(load(q), E);
    __syncthreads();
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) {
        const int i = q % NP, j = (q / NP) % NP, k = q / NP2;
        dfacc ar = df_mul(sDT[i], su[(k * NP + j) * NP]);
        dfacc as = df_mul(sDT[j], su[k * NP2 + i]);
        dfacc at = df_mul(sDT[k], su[j * NP + i]);
        for (int l = 1; l < NP; ++l) {
            df_mad(ar, sDT[l * NP + i], su[(k * NP + j) * NP + l]);
            df_mad(as, sDT[l * NP + j], su[(k * NP + l) * NP + i]);
            df_mad(at, sDT[l * NP + k], su[(l * NP + j) * NP + i]);
        }
        const dfp ur = df_raw(ar), us = df_raw(as), ut = df_raw(at);
        const dfp g11 = geo[0 * NP3 + q], g22 = geo[1 * NP3 + q], g33 = geo[2 * NP3 + q];
        const dfp g12 = geo[3 * NP3 + q], g13 = geo[4 * NP3 + q], g23 = geo[5 * NP3 + q];
        dfacc vr = df_mul(g11, ur), vs = df_mul(g12, ur), vt = df_mul(g13, ur);
        df_mad(vr, g12, us); df_mad(vr, g13, ut);
        df_mad(vs, g22, us); df_mad(vs, g23, ut);
        df_mad(vt, g23, us); df_mad(vt, g33, ut);
        svr[q] = df_raw(vr);
        svs[q] = df_raw(vs);
        svt[q] = df_raw(vt);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) {
        const int i = q % NP, j = (q / NP) % NP, k = q / NP2;
        dfacc ar = df_mul(sD[i], svr[(k * NP + j) * NP]);
        dfacc as = df_mul(sD[j], svs[k * NP2 + i]);
        dfacc at = df_mul(sD[k], svt[j * NP + i]);
        for (int l = 1; l < NP; ++l) {
            df_mad(ar, sD[l * NP + i], svr[(k * NP + j) * NP + l]);
            df_mad(as, sD[l * NP + j], svs[(k * NP + l) * NP + i]);
            df_mad(at, sD[l * NP + k], svt[(l * NP + j) * NP + i]);
        }
        df_add(ar, df_raw(as));
        df_add(ar, df_raw(at));
        const dfacc bu = df_mul(geo[6 * NP3 + q], su[q]);
        dfacc o = df_mul(h1, df_raw(ar));
        df_mad(o, h2, df_raw(bu));
        store(q, df_join_scaled(df_raw(o), E));
    }
    __syncthreads();
}
