// solve_np04.cu -- persistent solver kernels for order N = 3 (up to 8 problems).
#include "solver.cuh"

int sem_solve_launch_np4(const SolveParams<8> &p, int mode, int sms, long long mi, cudaStream_t s)
{
    switch (mode) {
        case MODE_F64: return launch_solve<8, MODE_F64, 4>(p, sms, mi, s);
        case MODE_F64N: return launch_solve<8, MODE_F64N, 4>(p, sms, mi, s);
        case MODE_F32: return launch_solve<8, MODE_F32, 4>(p, sms, mi, s);
        case MODE_TC: return launch_solve<8, MODE_TC, 4>(p, sms, mi, s);
        default: return SEM_ERR_ARG;
    }
}

int sem_solve_tables_np4(const void *tabs) { return solver_upload_bfp_tables(4, tabs); }
