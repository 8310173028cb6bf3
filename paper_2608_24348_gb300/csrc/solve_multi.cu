// solve_multi.cu -- persistent solver kernels for batches mixing N = 5, 7, 9.
#include "solver.cuh"

int sem_solve_launch_multi(const SolveParams<SEM_MAXP> &p, int mode, int sms, long long mi,
                           cudaStream_t s)
{
    switch (mode) {
        case MODE_F64: return launch_solve<SEM_MAXP, MODE_F64, 6, 8, 10>(p, sms, mi, s);
        case MODE_F32: return launch_solve<SEM_MAXP, MODE_F32, 6, 8, 10>(p, sms, mi, s);
        case MODE_TC: return launch_solve<SEM_MAXP, MODE_TC, 6, 8, 10>(p, sms, mi, s);
        case MODE_F64N: return launch_solve<SEM_MAXP, MODE_F64N, 6, 8, 10>(p, sms, mi, s);
        default: return SEM_ERR_ARG;
    }
}

int sem_solve_tables_multi(int np, const void *tabs) { return solver_upload_bfp_tables(np, tabs); }
