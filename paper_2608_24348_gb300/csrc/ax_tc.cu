// ax_tc.cu -- element operator with 16-bit tensor-core contractions.
#include "common.cuh"

int sem_ax_tc(sem_ctx *, const float *, float *, double, double, int, cudaStream_t)
{
    return SEM_ERR_ARG;
}
