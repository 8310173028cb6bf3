// ax_f32.cu -- F32 instantiations of the stand-alone element operator.
#include "ax_launch.cuh"

int sem_launch_ax_f32(const sem_ctx *c, const float *u, float *w, float h1, float h2, cudaStream_t s)
{
    const int n = c->n;
    const float *tab = c->tab32 + 2 * n;
    const float *geo = c->geo32;
    SEM_DISPATCH_NP(n, return launch_ax<NP, float>(c, u, w, geo, tab, h1, h2, s));
    return SEM_ERR_ARG;
}
