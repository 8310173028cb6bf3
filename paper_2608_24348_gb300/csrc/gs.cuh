// gs.cuh -- index arithmetic of the structured-box gather-scatter.
//
// Unique node g = gx + ngx (gy + ngy gz).  Along one direction with nel
// elements of order N, unique index gd lies inside element gd / N at local
// index gd % N, and when gd % N == 0 it is also the last node (local index N)
// of the previous element (wrapping around in a periodic direction).  Shared
// nodes therefore have 2, 4 or 8 copies; nodes inside an element have one.
#pragma once

#include <stdint.h>

struct GsDesc {
    int N, n, nelx, nely, nelz;
    int ngx, ngy, ngz;
    int px, py, pz;
    int64_t nG;
};

// Copies of unique index g along one direction: (element, local index).
__device__ __forceinline__ int gs_copies_1d(int g, int N, int nel, int periodic, int ce[2],
                                            int ci[2])
{
    int e = g / N;
    int i = g - e * N;
    if (i != 0) {
        ce[0] = e;
        ci[0] = i;
        return 1;
    }
    if (periodic) {
        ce[0] = e;
        ci[0] = 0;
        ce[1] = (e == 0) ? nel - 1 : e - 1;
        ci[1] = N;
        return 2;
    }
    int m = 0;
    if (e < nel) { ce[m] = e; ci[m] = 0; ++m; }
    if (e > 0) { ce[m] = e - 1; ci[m] = N; ++m; }
    return m;
}

// Local node indices of all copies of unique node g; returns the count (1..8).
__device__ __forceinline__ int gs_copies(const GsDesc &d, int64_t g, int64_t idx[8])
{
    int gx = (int)(g % d.ngx);
    int64_t t = g / d.ngx;
    int gy = (int)(t % d.ngy);
    int gz = (int)(t / d.ngy);
    int ex[2], ix[2], ey[2], iy[2], ez[2], iz[2];
    int mx = gs_copies_1d(gx, d.N, d.nelx, d.px, ex, ix);
    int my = gs_copies_1d(gy, d.N, d.nely, d.py, ey, iy);
    int mz = gs_copies_1d(gz, d.N, d.nelz, d.pz, ez, iz);
    int m = 0;
    const int n = d.n;
    for (int c = 0; c < mz; ++c)
        for (int b = 0; b < my; ++b)
            for (int a = 0; a < mx; ++a) {
                int64_t e = ex[a] + (int64_t)d.nelx * (ey[b] + (int64_t)d.nely * ez[c]);
                idx[m++] = e * (int64_t)(n * n * n) + (iz[c] * n + iy[b]) * n + ix[a];
            }
    return m;
}

// Multiplicity of local node (i, j, k) of element (ex, ey, ez).
__device__ __forceinline__ int gs_mult_local(const GsDesc &d, int ex, int ey, int ez, int i, int j,
                                             int k)
{
    int m = 1;
    if ((i == 0 && (d.px || ex > 0)) || (i == d.N && (d.px || ex < d.nelx - 1))) m *= 2;
    if ((j == 0 && (d.py || ey > 0)) || (j == d.N && (d.py || ey < d.nely - 1))) m *= 2;
    if ((k == 0 && (d.pz || ez > 0)) || (k == d.N && (d.pz || ez < d.nelz - 1))) m *= 2;
    return m;
}
