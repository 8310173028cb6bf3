// solve_np09.cu -- persistent solver kernels for order N = 8 (up to 8 problems).
#include "solver.cuh"

int sem_solve_launch_np9(const SolveParams<8> &p, int mode, int sms, long long mi, cudaStream_t s)
{
    switch (mode) {
        case MODE_F64: return launch_solve<8, MODE_F64, 9>(p, sms, mi, s);
        case MODE_F64N: return launch_solve<8, MODE_F64N, 9>(p, sms, mi, s);
        case MODE_F32: return launch_solve<8, MODE_F32, 9>(p, sms, mi, s);
        case MODE_TC: return launch_solve<8, MODE_TC, 9>(p, sms, mi, s);
        default: return SEM_ERR_ARG;
    }
}
