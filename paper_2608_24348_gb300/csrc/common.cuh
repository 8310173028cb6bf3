// common.cuh -- internal definitions shared by the libsem translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "sem.h"

#define SEM_NMAX 15
#define SEM_NPMAX 16

// Per-thread last CUDA error, reported by sem_last_cuda_error().
void sem_note_cuda_error(cudaError_t e, const char *where);

#define SEM_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            sem_note_cuda_error(e_, #call);                                             \
            return SEM_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

#define SEM_CHECK_LAUNCH()                                                              \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess) {                                                        \
            sem_note_cuda_error(e_, "kernel launch");                                   \
            return SEM_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

// One PCG workspace: the vectors of a solve (FP64 and FP32 sets).
struct sem_ws {
    double *r, *p, *w, *minv, *b;   // FP64 E-vectors (b: mean-free scratch copy is not kept)
    float *r32, *p32, *w32, *d32, *minv32;
    // minv (and minv32) hold the Jacobi inverse of (jac_h1, jac_h2) when jac_ok (jac32_ok)
    double jac_h1, jac_h2;
    int jac_ok, jac32_ok;
};

struct sem_ctx {
    int N, n, nelx, nely, nelz;
    int periodic[3];
    int64_t E, nL, nG;
    int ngx, ngy, ngz;
    double L[3];
    double volume;
    int device, num_sms;
    // 1-D tables on the device: xi[n], w[n], D[n*n] (row-major D_ij = l_j'(xi_i))
    double *tab64;
    float *tab32;
    double hD[SEM_NPMAX * SEM_NPMAX], hxi[SEM_NPMAX], hw[SEM_NPMAX];
    // geometry, element-blocked [E][7][n^3]: G11 G22 G33 G12 G13 G23 B
    double *geo64;
    float *geo32;
    void *geodf;       // float pairs of geo64 (FP64-accurate operator on FP32 pipes)
    void *tabdf;       // float pairs of D
    void *tabdfeo;     // float pairs of the folded half tables (even N+1)
    void *bfp_tabs;    // host copy of the block-floating-point kernel's tables (even N+1)
    double *vert;      // device vertex grid [(nelz+1)(nely+1)(nelx+1)][3]
    double *jinv64;    // [E][9][n^3] dr_a/dx_c at a*3+c (allocated by the stepper)
    float *jinv32;
    // solver workspaces (slot 0 allocated at setup)
    int nws;              // (unused)
    sem_ws ws[8];         // 0-3: solves through the API; 4-7: the Taylor-Green stepper's own
                          // (allocated on first use; a slot is allocated when its r is set)
    // device-side solve state + pinned host mirror of the last solve's info
    void *solve_dev;      // sem_solve_state[1]
    void *solve_host;     // pinned
    void *partials;       // reduction partials (device)
    size_t partials_bytes;
    // error word of bounded waits in stand-alone kernels (SEM_OK or SEM_ERR_TIMEOUT)
    void *err_dev;
    // host-pointer staging
    void *stage[2];
    size_t stage_bytes;
    void *pipe;           // streams and events of the pipelined host-buffer sem_ax (lazy)
    int u_sysmem;         // sem_ax's u is mapped host memory: no L2 bulk prefetch of it
};

static inline int64_t sem_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Raises a kernel's dynamic shared-memory limit to smem once per device: done
// holds one bit per device ordinal (0..31) and is set only after success, so
// concurrent first calls at worst both set the attribute.
template <class K>
static inline cudaError_t sem_smem_attr(K *kernel, size_t smem, std::atomic<unsigned> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = 1u << (dev & 31);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// ---------------------------------------------------------------------------
// Compile-time dispatch on NP = N + 1
// ---------------------------------------------------------------------------
#define SEM_NP_CASE(NPV, ...) \
    case NPV: {               \
        constexpr int NP = NPV; \
        __VA_ARGS__;          \
    } break;

#define SEM_DISPATCH_NP(npval, ...)                                                      \
    switch (npval) {                                                                     \
        SEM_NP_CASE(2, __VA_ARGS__)                                                      \
        SEM_NP_CASE(3, __VA_ARGS__)                                                      \
        SEM_NP_CASE(4, __VA_ARGS__)                                                      \
        SEM_NP_CASE(5, __VA_ARGS__)                                                      \
        SEM_NP_CASE(6, __VA_ARGS__)                                                      \
        SEM_NP_CASE(7, __VA_ARGS__)                                                      \
        SEM_NP_CASE(8, __VA_ARGS__)                                                      \
        SEM_NP_CASE(9, __VA_ARGS__)                                                      \
        SEM_NP_CASE(10, __VA_ARGS__)                                                     \
        SEM_NP_CASE(11, __VA_ARGS__)                                                     \
        SEM_NP_CASE(12, __VA_ARGS__)                                                     \
        SEM_NP_CASE(13, __VA_ARGS__)                                                     \
        SEM_NP_CASE(14, __VA_ARGS__)                                                     \
        SEM_NP_CASE(15, __VA_ARGS__)                                                     \
        SEM_NP_CASE(16, __VA_ARGS__)                                                     \
        default: return SEM_ERR_ARG;                                                     \
    }

// Host-pointer staging: returns a device pointer for `p` (p itself when it is
// device memory).  For inputs (copy_in) host data is copied into staging slot
// `slot`; outputs are copied back by sem_stage_out.
int sem_stage_in(sem_ctx *ctx, const void *p, size_t bytes, int slot, cudaStream_t s,
                 const void **dev, int *is_host);
int sem_stage_out_ptr(sem_ctx *ctx, void *p, size_t bytes, int slot, void **dev, int *is_host);
int sem_is_device_ptr(const void *p);
// the stand-alone operator's tile-shape candidate in force for order N and dtype
int sem_ax_variant(int N, sem_dtype dt);
