// ax_dfeo.cuh -- FP64-accurate element operator with folded (even-odd) contractions.
//
// The GLL derivative matrix is centro-antisymmetric, D[NP-1-i][NP-1-l] = -D[i][l]
// (also D^T).  With H = NP/2 (NP even), the even and odd parts of a line,
//     e_l = u_l + u_{NP-1-l},   o_l = u_l - u_{NP-1-l}     (l < H),
// and the half matrices A_il = (D_il + D_{i,NP-1-l})/2, B_il = (D_il - D_{i,NP-1-l})/2,
// every output pair of a 1-D contraction follows from two half-length sums:
//     a_i = sum_l A_il e_l,  b_i = sum_l B_il o_l,
//     (Du)_i = a_i + b_i,    (Du)_{NP-1-i} = b_i - a_i          (i < H),
// which halves the multiply-adds of all six directional contractions.  The
// arithmetic is the float-pair compensated arithmetic of ax_df.cuh; pairs pass
// between stages without renormalisation.
//
// Thread (i, j) of an element owns column u[.][j][i] (the t direction stays in
// registers).  For r and s it folds one line of each direction into shared
// memory, then computes the output pairs of H lines; results return to the
// column owner through shared memory.  Shared memory per element: five
// float-pair slabs of NP^2 lines, each line padded to NP+1 entries so that 32
// threads reading 32 different lines at the same offset hit distinct banks.
#pragma once

#include "ax_df.cuh"

template <int NP>
struct AxEoCfg {
    static constexpr int H = NP / 2;
    static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    static constexpr int NE = (256 / NP2) > 0 ? (256 / NP2) : 1;
    static constexpr int THREADS = NE * NP2;
    static constexpr bool OK = (NP % 2) == 0;
    static constexpr int LS = NP + 1;           // padded line stride of a slab
    static constexpr int SLAB = NP2 * LS;       // float pairs per slab
};

// Half tables: A, B of D (gradient) and AT, BT of D^T (transpose), H*H each,
// then NE elements' slabs and exponents.
template <int NP, int NE>
__host__ __device__ constexpr size_t ax_dfeo_smem_bytes_ne()
{
    return sizeof(dfp) * (4 * (NP / 2) * (NP / 2) + (size_t)NE * 5 * NP * NP * (NP + 1)) + sizeof(int) * NE;
}

template <int NP>
__host__ __device__ constexpr size_t ax_dfeo_smem_bytes()
{
    return ax_dfeo_smem_bytes_ne<NP, AxEoCfg<NP>::NE>();
}

__device__ __forceinline__ dfp df_neg(dfp a) { return {-a.hi, -a.lo}; }

// Synchronisation between the stages of one element: GS == 0 is the block
// barrier; GS > 0 is hardware barrier 1 + grp counted over the GS threads of
// element group grp only (GS a multiple of 32; every thread of the group
// reaches the same barriers), so the element groups of a block need not move
// in step.
template <int GS>
__device__ __forceinline__ void dfeo_sync(int grp)
{
    if constexpr (GS == 0) {
        __syncthreads();
    } else {
        static_assert(GS % 32 == 0, "a named barrier counts whole warps");
        asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "n"(GS) : "memory");
    }
}

// tab: the four half tables laid out [A | B | AT | BT], each H*H row-major [i][l],
// loaded and published before the first call.
template <int NP, int GS = 0, class Load, class Store>
__device__ __forceinline__ void ax_dfeo_element(const Load &load, const Store &store,
                                                const dfp *__restrict__ geo, dfp h1, dfp h2,
                                                const dfp *__restrict__ tab, dfp *__restrict__ slab,
                                                int *sexp, int tid, bool active, int grp = 0)
{
    constexpr int H = NP / 2, NP2 = NP * NP, NP3 = NP2 * NP, HH = H * H;
    constexpr int LS = AxEoCfg<NP>::LS, SL = AxEoCfg<NP>::SLAB;
    const dfp *tA = tab, *tB = tab + HH, *tAT = tab + 2 * HH, *tBT = tab + 3 * HH;
    dfp *su = slab, *f1 = slab + SL, *f2 = f1 + SL, *g1 = f2 + SL, *g2 = g1 + SL;
    const int i = tid % NP, j = tid / NP;
    // ---- load, element exponent, split
    double xu[NP];
    if (tid == 0) *sexp = 0;
    dfeo_sync<GS>(grp);
    if (active) {
        int m = 0;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            xu[k] = load(k * NP2 + tid);
            m = max(m, df_bexp(xu[k]));
        }
        atomicMax(sexp, m);
    }
    dfeo_sync<GS>(grp);
    const int E = *sexp > 0 ? *sexp - 1023 : 0;
    dfp ru[NP];
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            ru[k] = df_split_scaled(xu[k], E);
            su[(k * NP + j) * LS + i] = ru[k];
        }
    }
    dfeo_sync<GS>(grp);
    // ---- fold the r-line (k = j, row i) into f1 and the s-line (k = j, column i) into f2
    if (active) {
        const dfp *lr = su + (j * NP + i) * LS;
        dfp *fr = f1 + (j * NP + i) * LS;
#pragma unroll
        for (int l = 0; l < H; ++l) {
            const dfp a = lr[l], b = lr[NP - 1 - l];
            fr[l] = df_sum(a, b);
            fr[H + l] = df_sum(a, df_neg(b));
        }
#pragma unroll
        for (int l = 0; l < H; ++l) {
            const dfp a = su[(j * NP + l) * LS + i], b = su[(j * NP + NP - 1 - l) * LS + i];
            f2[(j * NP + l) * LS + i] = df_sum(a, b);
            f2[(j * NP + H + l) * LS + i] = df_sum(a, df_neg(b));
        }
    }
    dfeo_sync<GS>(grp);
    // ---- gradient: r pairs -> g1, s pairs -> g2, t in registers
    dfp ut[NP];
    if (active) {
        const int ip = i % H, kr = (i / H) * H;
#pragma unroll
        for (int kk = 0; kk < H; ++kk) {
            const int k = kr + kk;
            const dfp *fr = f1 + (k * NP + j) * LS;
            dfacc a = df_mul(tA[ip * H], fr[0]), b = df_mul(tB[ip * H], fr[H]);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                df_mad(a, tA[ip * H + l], fr[l]);
                df_mad(b, tB[ip * H + l], fr[H + l]);
            }
            const dfp av = df_raw(a), bv = df_raw(b);
            g1[(k * NP + j) * LS + ip] = df_sum(av, bv);
            g1[(k * NP + j) * LS + NP - 1 - ip] = df_sum(bv, df_neg(av));
        }
        const int jp = j % H, ks = (j / H) * H;
#pragma unroll
        for (int kk = 0; kk < H; ++kk) {
            const int k = ks + kk;
            dfacc a = df_mul(tA[jp * H], f2[(k * NP) * LS + i]);
            dfacc b = df_mul(tB[jp * H], f2[(k * NP + H) * LS + i]);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                df_mad(a, tA[jp * H + l], f2[(k * NP + l) * LS + i]);
                df_mad(b, tB[jp * H + l], f2[(k * NP + H + l) * LS + i]);
            }
            const dfp av = df_raw(a), bv = df_raw(b);
            g2[(k * NP + jp) * LS + i] = df_sum(av, bv);
            g2[(k * NP + NP - 1 - jp) * LS + i] = df_sum(bv, df_neg(av));
        }
        dfp e[H], o[H];
#pragma unroll
        for (int l = 0; l < H; ++l) {
            e[l] = df_sum(ru[l], ru[NP - 1 - l]);
            o[l] = df_sum(ru[l], df_neg(ru[NP - 1 - l]));
        }
#pragma unroll
        for (int kp = 0; kp < H; ++kp) {
            dfacc a = df_mul(tA[kp * H], e[0]), b = df_mul(tB[kp * H], o[0]);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                df_mad(a, tA[kp * H + l], e[l]);
                df_mad(b, tB[kp * H + l], o[l]);
            }
            const dfp av = df_raw(a), bv = df_raw(b);
            ut[kp] = df_sum(av, bv);
            ut[NP - 1 - kp] = df_sum(bv, df_neg(av));
        }
    }
    dfeo_sync<GS>(grp);
    // ---- geometric factors (column owner): vr -> f1, vs -> f2, vt in registers
    dfp rw[NP];
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = k * NP2 + tid, q = (k * NP + j) * LS + i;
            const dfp ur = g1[q], us = g2[q];
            const dfp g11 = geo[0 * NP3 + p], g22 = geo[1 * NP3 + p], g33 = geo[2 * NP3 + p];
            const dfp g12 = geo[3 * NP3 + p], g13 = geo[4 * NP3 + p], g23 = geo[5 * NP3 + p];
            const dfp bm = geo[6 * NP3 + p];
            dfacc vr = df_mul(g11, ur), vs = df_mul(g12, ur), vt = df_mul(g13, ur);
            df_mad(vr, g12, us); df_mad(vr, g13, ut[k]);
            df_mad(vs, g22, us); df_mad(vs, g23, ut[k]);
            df_mad(vt, g23, us); df_mad(vt, g33, ut[k]);
            const dfacc vw = df_mul(bm, ru[k]);
            f1[q] = df_raw(vr);
            f2[q] = df_raw(vs);
            ut[k] = df_raw(vt);  // ut now holds vt of this column
            rw[k] = df_raw(vw);
        }
    }
    dfeo_sync<GS>(grp);
    // ---- fold vr (r-line k = j, row i) into g1, vs (s-line k = j, column i) into g2
    if (active) {
        const dfp *lr = f1 + (j * NP + i) * LS;
        dfp *fr = g1 + (j * NP + i) * LS;
#pragma unroll
        for (int l = 0; l < H; ++l) {
            const dfp a = lr[l], b = lr[NP - 1 - l];
            fr[l] = df_sum(a, b);
            fr[H + l] = df_sum(a, df_neg(b));
        }
#pragma unroll
        for (int l = 0; l < H; ++l) {
            const dfp a = f2[(j * NP + l) * LS + i], b = f2[(j * NP + NP - 1 - l) * LS + i];
            g2[(j * NP + l) * LS + i] = df_sum(a, b);
            g2[(j * NP + H + l) * LS + i] = df_sum(a, df_neg(b));
        }
    }
    dfeo_sync<GS>(grp);
    // ---- transpose: r pairs -> f1, s pairs -> f2, t in registers
    dfp wt[NP];
    if (active) {
        const int ip = i % H, kr = (i / H) * H;
#pragma unroll
        for (int kk = 0; kk < H; ++kk) {
            const int k = kr + kk;
            const dfp *fr = g1 + (k * NP + j) * LS;
            dfacc a = df_mul(tAT[ip * H], fr[0]), b = df_mul(tBT[ip * H], fr[H]);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                df_mad(a, tAT[ip * H + l], fr[l]);
                df_mad(b, tBT[ip * H + l], fr[H + l]);
            }
            const dfp av = df_raw(a), bv = df_raw(b);
            f1[(k * NP + j) * LS + ip] = df_sum(av, bv);
            f1[(k * NP + j) * LS + NP - 1 - ip] = df_sum(bv, df_neg(av));
        }
        const int jp = j % H, ks = (j / H) * H;
#pragma unroll
        for (int kk = 0; kk < H; ++kk) {
            const int k = ks + kk;
            dfacc a = df_mul(tAT[jp * H], g2[(k * NP) * LS + i]);
            dfacc b = df_mul(tBT[jp * H], g2[(k * NP + H) * LS + i]);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                df_mad(a, tAT[jp * H + l], g2[(k * NP + l) * LS + i]);
                df_mad(b, tBT[jp * H + l], g2[(k * NP + H + l) * LS + i]);
            }
            const dfp av = df_raw(a), bv = df_raw(b);
            f2[(k * NP + jp) * LS + i] = df_sum(av, bv);
            f2[(k * NP + NP - 1 - jp) * LS + i] = df_sum(bv, df_neg(av));
        }
        dfp e[H], o[H];
#pragma unroll
        for (int l = 0; l < H; ++l) {
            e[l] = df_sum(ut[l], ut[NP - 1 - l]);
            o[l] = df_sum(ut[l], df_neg(ut[NP - 1 - l]));
        }
#pragma unroll
        for (int kp = 0; kp < H; ++kp) {
            dfacc a = df_mul(tAT[kp * H], e[0]), b = df_mul(tBT[kp * H], o[0]);
#pragma unroll
            for (int l = 1; l < H; ++l) {
                df_mad(a, tAT[kp * H + l], e[l]);
                df_mad(b, tBT[kp * H + l], o[l]);
            }
            const dfp av = df_raw(a), bv = df_raw(b);
            wt[kp] = df_sum(av, bv);
            wt[NP - 1 - kp] = df_sum(bv, df_neg(av));
        }
    }
    dfeo_sync<GS>(grp);
    // ---- sum of the three directions, h1 / h2 weights, rounding to FP64
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = k * NP2 + tid, q = (k * NP + j) * LS + i;
            dfacc s = {wt[k].hi, wt[k].lo};
            df_add(s, f1[q]);
            df_add(s, f2[q]);
            dfacc o = df_mul(h1, df_raw(s));
            df_mad(o, h2, rw[k]);
            store(p, df_join_scaled(df_raw(o), E));
        }
    }
    dfeo_sync<GS>(grp);
}

// Host: the four half tables from the FP64 derivative matrix D (row-major n x n).
static inline void ax_dfeo_tables(int n, const double *D, dfp *out)
{
    const int H = n / 2, HH = H * H;
    for (int i = 0; i < H; ++i)
        for (int l = 0; l < H; ++l) {
            const double a = 0.5 * (D[i * n + l] + D[i * n + n - 1 - l]);
            const double b = 0.5 * (D[i * n + l] - D[i * n + n - 1 - l]);
            const double at = 0.5 * (D[l * n + i] + D[(n - 1 - l) * n + i]);
            const double bt = 0.5 * (D[l * n + i] - D[(n - 1 - l) * n + i]);
            const double v[4] = {a, b, at, bt};
            for (int t = 0; t < 4; ++t) {
                const float h = (float)v[t];
                out[t * HH + i * H + l] = {h, (float)(v[t] - (double)h)};
            }
        }
}
