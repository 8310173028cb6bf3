// solve_np08.cu -- persistent solver kernels for order N = 7 (up to 8 problems).
#include "solver.cuh"

int sem_solve_launch_np8(const SolveParams<8> &p, int mode, int sms, long long mi, cudaStream_t s)
{
    switch (mode) {
        case MODE_F64: return launch_solve<8, MODE_F64, 8>(p, sms, mi, s);
        case MODE_F64N: return launch_solve<8, MODE_F64N, 8>(p, sms, mi, s);
        case MODE_F32: return launch_solve<8, MODE_F32, 8>(p, sms, mi, s);
        case MODE_TC: return launch_solve<8, MODE_TC, 8>(p, sms, mi, s);
        default: return SEM_ERR_ARG;
    }
}

int sem_solve_tables_np8(const void *tabs) { return solver_upload_bfp_tables(8, tabs); }
