// ax_f64.cu -- F64 instantiations of the stand-alone element operator.
#include "ax_launch.cuh"

int sem_launch_ax_f64(const sem_ctx *c, const double *u, double *w, double h1, double h2, cudaStream_t s)
{
    const int n = c->n;
    const double *tab = c->tab64 + 2 * n;
    const double *geo = c->geo64;
    SEM_DISPATCH_NP(n, return launch_ax<NP, double>(c, u, w, geo, tab, h1, h2, s));
    return SEM_ERR_ARG;
}
