// solve_np16.cu -- persistent solver kernels for order N = 15 (up to 8 problems).
#include "solver.cuh"

int sem_solve_launch_np16(const SolveParams<8> &p, int mode, int sms, long long mi, cudaStream_t s)
{
    switch (mode) {
        case MODE_F64: return launch_solve<8, MODE_F64, 16>(p, sms, mi, s);
        case MODE_F64N: return launch_solve<8, MODE_F64N, 16>(p, sms, mi, s);
        case MODE_F32: return launch_solve<8, MODE_F32, 16>(p, sms, mi, s);
        case MODE_TC: return SEM_ERR_ARG;
        default: return SEM_ERR_ARG;
    }
}

int sem_solve_tables_np16(const void *tabs) { return solver_upload_bfp_tables(16, tabs); }
