// tgv.cu -- Taylor-Green vortex stepper (BDF3/EXT3 P_N-P_N, 3/2 dealiasing).
#include "common.cuh"

extern "C" int sem_tgv_init(sem_ctx *, double, double, sem_dtype, const sem_solve_opts *,
                            const sem_solve_opts *, sem_tgv **out)
{
    if (out) *out = nullptr;
    return SEM_ERR_ARG;
}
extern "C" int sem_tgv_set(sem_tgv *, int, const double *, const double *, const double *,
                           const double *, int, double, void *)
{
    return SEM_ERR_ARG;
}
extern "C" int sem_tgv_step(sem_tgv *, int, sem_tgv_diag *, void *) { return SEM_ERR_ARG; }
extern "C" int sem_tgv_get(sem_tgv *, double *, double *, double *, double *, void *)
{
    return SEM_ERR_ARG;
}
extern "C" int sem_tgv_energy(sem_tgv *, double *, double *, void *) { return SEM_ERR_ARG; }
extern "C" void sem_tgv_destroy(sem_tgv *) {}
