// solve_np04.cu -- persistent solver kernel for order N = 3 (up to 8 problems).
#include "solver.cuh"

int sem_solve_launch_np4(const SolveParams<8> &p, int sms, long long mi, cudaStream_t s)
{
    return launch_solve<8, 4>(p, sms, mi, s);
}
