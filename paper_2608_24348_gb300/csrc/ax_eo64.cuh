// ax_eo64.cuh -- the native FP64 element operator with folded (even-odd)
// contractions.
//
// The GLL derivative matrix is centro-antisymmetric, D[N-i][N-l] = -D[i][l].
// With H = NP/2 (NP even) and the even / odd parts of a line
//     e_l = u_l + u_{N-l},   o_l = u_l - u_{N-l}          (l < H),
// the half matrices A_il = (D_il + D_{i,N-l})/2, B_il = (D_il - D_{i,N-l})/2
// give each output pair of a 1-D contraction from two half-length sums:
//     a_i = sum_l A_il e_l,  b_i = sum_l B_il o_l,
//     (Du)_i = a_i + b_i,    (Du)_{N-i} = b_i - a_i       (i < H);
// likewise for D^T with the transposed half matrices.  A line costs NP*H fused
// multiply-adds instead of NP*NP, plus NP additions for the fold and NP for
// the output pairs: about 6 FP64 operations per node and direction instead of
// 8 at NP = 8.
//
// Thread (i, j) of an element owns column u[.][j][i] (the t direction in
// registers).  It folds the r line (k' = j, j' = i) and the s line (k' = j,
// i' = i) into shared memory, then computes the output pairs (i mod H) of H r
// lines and (j mod H) of H s lines; the results return to the column owners
// through shared memory.  Five slabs of NP^2 lines per element, each line
// padded to NP+1 doubles.
#pragma once

#include "common.cuh"

template <int NP>
struct AxEo64Cfg {
    static constexpr int H = NP / 2;
    static constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
    static constexpr int NE = (256 / NP2) > 0 ? (256 / NP2) : 1;
    static constexpr int THREADS = NE * NP2;
    static constexpr int LS = NP + 1;
    static constexpr int SLAB = NP2 * LS;
};

// Shared memory: the four half tables [A | B | AT | BT] (H*H each), then NE
// elements' five slabs.
template <int NP>
__host__ __device__ constexpr size_t ax_eo64_smem_bytes()
{
    using C = AxEo64Cfg<NP>;
    return sizeof(double) * (4 * C::H * C::H + (size_t)C::NE * 5 * C::SLAB);
}

// Host: the half tables from D (row-major n x n, D_ij = l_j'(xi_i)).
static inline void ax_eo64_tables(int n, const double *D, double *out)
{
    const int H = n / 2, HH = H * H;
    for (int i = 0; i < H; ++i)
        for (int l = 0; l < H; ++l) {
            out[0 * HH + i * H + l] = 0.5 * (D[i * n + l] + D[i * n + n - 1 - l]);
            out[1 * HH + i * H + l] = 0.5 * (D[i * n + l] - D[i * n + n - 1 - l]);
            out[2 * HH + i * H + l] = 0.5 * (D[l * n + i] + D[(n - 1 - l) * n + i]);
            out[3 * HH + i * H + l] = 0.5 * (D[l * n + i] - D[(n - 1 - l) * n + i]);
        }
}

// Fold a line that runs along the fastest index of slab `src` (r line) and one
// that runs along the middle index (s line) into `dr`, `ds`: entries l < H hold
// e_l, entries H + l hold o_l, in the same line positions.
template <int NP>
__device__ __forceinline__ void eo64_fold(const double *src_r, const double *src_s, double *dr, double *ds,
                                          int i, int j)
{
    constexpr int H = NP / 2, LS = NP + 1;
    const double *lr = src_r + (j * NP + i) * LS;
    double *fr = dr + (j * NP + i) * LS;
#pragma unroll
    for (int l = 0; l < H; ++l) {
        const double a = lr[l], b = lr[NP - 1 - l];
        fr[l] = a + b;
        fr[H + l] = a - b;
    }
#pragma unroll
    for (int l = 0; l < H; ++l) {
        const double a = src_s[(j * NP + l) * LS + i], b = src_s[(j * NP + NP - 1 - l) * LS + i];
        ds[(j * NP + l) * LS + i] = a + b;
        ds[(j * NP + H + l) * LS + i] = a - b;
    }
}

// Output pairs of the folded r lines (k, j), k in thread i's range, into `gr`,
// and of the folded s lines (k, i), k in thread j's range, into `gs`; tA, tB
// the half tables of the contraction (D or D^T).
template <int NP>
__device__ __forceinline__ void eo64_pairs(const double *fr_slab, const double *fs_slab, double *gr, double *gs,
                                           const double *tA, const double *tB, int i, int j)
{
    constexpr int H = NP / 2, LS = NP + 1;
    const int ip = i % H, kr = (i / H) * H;
#pragma unroll
    for (int kk = 0; kk < H; ++kk) {
        const int k = kr + kk;
        const double *fr = fr_slab + (k * NP + j) * LS;
        double a = tA[ip * H] * fr[0], b = tB[ip * H] * fr[H];
#pragma unroll
        for (int l = 1; l < H; ++l) {
            a = fma(tA[ip * H + l], fr[l], a);
            b = fma(tB[ip * H + l], fr[H + l], b);
        }
        gr[(k * NP + j) * LS + ip] = a + b;
        gr[(k * NP + j) * LS + NP - 1 - ip] = b - a;
    }
    const int jp = j % H, ks = (j / H) * H;
#pragma unroll
    for (int kk = 0; kk < H; ++kk) {
        const int k = ks + kk;
        double a = tA[jp * H] * fs_slab[(k * NP) * LS + i], b = tB[jp * H] * fs_slab[(k * NP + H) * LS + i];
#pragma unroll
        for (int l = 1; l < H; ++l) {
            a = fma(tA[jp * H + l], fs_slab[(k * NP + l) * LS + i], a);
            b = fma(tB[jp * H + l], fs_slab[(k * NP + H + l) * LS + i], b);
        }
        gs[(k * NP + jp) * LS + i] = a + b;
        gs[(k * NP + NP - 1 - jp) * LS + i] = b - a;
    }
}

// t direction in registers: y = M x for the column x.
template <int NP>
__device__ __forceinline__ void eo64_column(const double (&x)[NP], double (&y)[NP], const double *tA,
                                            const double *tB)
{
    constexpr int H = NP / 2;
    double e[H], o[H];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        e[l] = x[l] + x[NP - 1 - l];
        o[l] = x[l] - x[NP - 1 - l];
    }
#pragma unroll
    for (int kp = 0; kp < H; ++kp) {
        double a = tA[kp * H] * e[0], b = tB[kp * H] * o[0];
#pragma unroll
        for (int l = 1; l < H; ++l) {
            a = fma(tA[kp * H + l], e[l], a);
            b = fma(tB[kp * H + l], o[l], b);
        }
        y[kp] = a + b;
        y[NP - 1 - kp] = b - a;
    }
}

// One element (all threads of the block call it; it synchronises the block).
// geo: the element's [7][NP^3] factors; tab: the four half tables in shared
// memory, published before the first call; slab: the element's five slabs.
template <int NP, class Load, class Store>
__device__ __forceinline__ void ax_eo64_element(const Load &load, const Store &store, const double *__restrict__ geo,
                                                double h1, double h2, const double *__restrict__ tab,
                                                double *__restrict__ slab, int tid, bool active)
{
    constexpr int H = NP / 2, NP2 = NP * NP, NP3 = NP2 * NP, HH = H * H;
    constexpr int LS = NP + 1, SL = NP2 * LS;
    const double *tA = tab, *tB = tab + HH, *tAT = tab + 2 * HH, *tBT = tab + 3 * HH;
    double *su = slab, *f1 = slab + SL, *f2 = f1 + SL, *g1 = f2 + SL, *g2 = g1 + SL;
    const int i = tid % NP, j = tid / NP;
    double ru[NP], ut[NP], rw[NP];
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            ru[k] = load(k * NP2 + tid);
            su[(k * NP + j) * LS + i] = ru[k];
        }
    }
    __syncthreads();
    if (active) eo64_fold<NP>(su, su, f1, f2, i, j);
    __syncthreads();
    if (active) {
        eo64_pairs<NP>(f1, f2, g1, g2, tA, tB, i, j);  // u_r -> g1, u_s -> g2
        eo64_column<NP>(ru, ut, tA, tB);                // u_t in registers
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int p = k * NP2 + tid, q = (k * NP + j) * LS + i;
            const double ur = g1[q], us = g2[q], uq = ut[k];
            const double g11 = geo[0 * NP3 + p], g22 = geo[1 * NP3 + p], g33 = geo[2 * NP3 + p];
            const double g12 = geo[3 * NP3 + p], g13 = geo[4 * NP3 + p], g23 = geo[5 * NP3 + p];
            f1[q] = fma(g11, ur, fma(g12, us, g13 * uq));
            f2[q] = fma(g12, ur, fma(g22, us, g23 * uq));
            ut[k] = fma(g13, ur, fma(g23, us, g33 * uq));  // ut now holds v_t of this column
            rw[k] = geo[6 * NP3 + p] * ru[k];
        }
    }
    __syncthreads();
    if (active) eo64_fold<NP>(f1, f2, g1, g2, i, j);
    __syncthreads();
    double wt[NP];
    if (active) {
        eo64_pairs<NP>(g1, g2, f1, f2, tAT, tBT, i, j);  // D_r^T v_r -> f1, D_s^T v_s -> f2
        eo64_column<NP>(ut, wt, tAT, tBT);
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int q = (k * NP + j) * LS + i;
            store(k * NP2 + tid, fma(h1, wt[k] + f1[q] + f2[q], h2 * rw[k]), ru[k]);
        }
    }
    __syncthreads();
}
