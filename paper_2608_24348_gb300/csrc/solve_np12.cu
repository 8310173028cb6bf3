// solve_np12.cu -- persistent solver kernel for order N = 11 (up to 8 problems).
#include "solver.cuh"

int sem_solve_launch_np12(const SolveParams<8> &p, int sms, long long mi, cudaStream_t s)
{
    return launch_solve<8, 12>(p, sms, mi, s);
}
