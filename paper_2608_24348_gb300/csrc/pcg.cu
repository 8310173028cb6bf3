// pcg.cu -- Jacobi PCG, FP64 iterative refinement, batched solves.
#include "common.cuh"

struct sem_solve_state {
    int status, iters, outer_iters, pad;
    double rnorm, bnorm;
};

int sem_solve_state_bytes() { return (int)sizeof(sem_solve_state) * 64; }

extern "C" void sem_solve_opts_default(sem_solve_opts *o)
{
    o->tol = 1e-10;
    o->abs_tol = 0;
    o->maxit = 20000;
    o->inner = SEM_F64;
    o->inner_tol = 1e-4;
    o->max_outer = 50;
}

extern "C" int sem_pcg_solve(sem_ctx *, const double *, double *, double, double,
                             const sem_solve_opts *, sem_solve_info *, void *)
{
    return SEM_ERR_ARG;
}

extern "C" int sem_last_solve_info(sem_ctx *, sem_solve_info *) { return SEM_ERR_ARG; }

extern "C" int sem_pcg_solve_batched(int, sem_ctx *const *, const double *const *, double *const *,
                                     const double *, const double *, const sem_solve_opts *,
                                     sem_solve_info *, void *)
{
    return SEM_ERR_ARG;
}
