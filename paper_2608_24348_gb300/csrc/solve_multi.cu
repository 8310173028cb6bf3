// solve_multi.cu -- persistent solver kernel for batches mixing N = 5, 7, 9.
#include "solver.cuh"

int sem_solve_launch_multi(const SolveParams<SEM_MAXP> &p, int sms, long long mi, cudaStream_t s)
{
    return launch_solve<SEM_MAXP, 6, 8, 10>(p, sms, mi, s);
}
