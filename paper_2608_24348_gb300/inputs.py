"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds no arithmetic of the method itself: only seeded random
draws (numpy PCG64), the vertex grid of a structured box, the index layout
that places a field given on unique grid points into the element-local
E-vector ``[E][N+1][N+1][N+1]`` (i fastest, e = ex + nelx*(ey + nely*ez)), and
analytic functions evaluated at caller-supplied coordinates.

Seeds: mesh 1, field 2, right-hand side 3, batch 4.
"""
from __future__ import annotations

import math

import numpy as np

SEED_MESH, SEED_FIELD, SEED_RHS, SEED_BATCH = 1, 2, 3, 4
TWO_PI = 2.0 * math.pi


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def box_vertices(nel, L=(TWO_PI, TWO_PI, TWO_PI), perturb=0.0, seed=SEED_MESH):
    """Vertex grid ``[(nelz+1), (nely+1), (nelx+1), 3]`` of a box [0,Lx]x[0,Ly]x[0,Lz].

    With ``perturb > 0`` every vertex whose three grid indices are all interior
    (1 <= I <= nelx-1, and likewise J, K) moves by an independent uniform draw
    in [-perturb*h, perturb*h] per coordinate (h = L/nel in that direction);
    draws are taken with I fastest, then J, then K, three (x, y, z) per vertex.
    Boundary planes stay flat, so a periodic identification stays a pure
    translation.
    """
    nx, ny, nz = (int(v) for v in nel)
    Lx, Ly, Lz = (float(v) for v in L)
    X = np.linspace(0.0, Lx, nx + 1)
    Y = np.linspace(0.0, Ly, ny + 1)
    Z = np.linspace(0.0, Lz, nz + 1)
    v = np.empty((nz + 1, ny + 1, nx + 1, 3))
    v[..., 0] = X[None, None, :]
    v[..., 1] = Y[None, :, None]
    v[..., 2] = Z[:, None, None]
    if perturb > 0 and nx > 1 and ny > 1 and nz > 1:
        d = _rng(seed).uniform(-1.0, 1.0, size=(nz - 1, ny - 1, nx - 1, 3))
        h = np.array([Lx / nx, Ly / ny, Lz / nz])
        v[1:nz, 1:ny, 1:nx, :] += perturb * h * d
    return v


def unique_counts(N, nel, periodic=(1, 1, 1)):
    """Number of unique grid points per direction."""
    return tuple(int(nel[d]) * N + (0 if periodic[d] else 1) for d in range(3))


def local_to_unique(N, nel, periodic=(1, 1, 1)):
    """Unique grid index (gx + ngx*(gy + ngy*gz)) of every local node, as an E-vector."""
    n = N + 1
    nx, ny, nz = (int(v) for v in nel)
    ngx, ngy, ngz = unique_counts(N, nel, periodic)
    # E-vector order [ez][ey][ex][k][j][i]
    k_ = np.arange(n).reshape(1, 1, 1, n, 1, 1)
    j_ = np.arange(n).reshape(1, 1, 1, 1, n, 1)
    i_ = np.arange(n).reshape(1, 1, 1, 1, 1, n)
    ex_ = np.arange(nx).reshape(1, 1, nx, 1, 1, 1)
    ey_ = np.arange(ny).reshape(1, ny, 1, 1, 1, 1)
    ez_ = np.arange(nz).reshape(nz, 1, 1, 1, 1, 1)
    gx = (ex_ * N + i_) % ngx
    gy = (ey_ * N + j_) % ngy
    gz = (ez_ * N + k_) % ngz
    g = gx + ngx * (gy + ngy * gz)
    return np.ascontiguousarray(g.reshape(-1)).astype(np.int64)


def unique_uniform_field(N, nel, periodic=(1, 1, 1), seed=SEED_FIELD, lo=-1.0, hi=1.0):
    """A field drawn U[lo, hi] once per unique grid point (gx fastest), laid out as
    an E-vector (shared nodes carry the same value: a continuous field)."""
    ngx, ngy, ngz = unique_counts(N, nel, periodic)
    ug = _rng(seed).uniform(lo, hi, size=ngx * ngy * ngz)
    return ug[local_to_unique(N, nel, periodic)]


def local_uniform_field(nL, seed=SEED_FIELD, lo=-1.0, hi=1.0):
    """A field drawn U[lo, hi] independently per local node (discontinuous)."""
    return _rng(seed).uniform(lo, hi, size=nL)


# ----------------------------------------------------------------------------
# Right-hand sides evaluated at given coordinates
# ----------------------------------------------------------------------------

def fourier_div_modes(seed=SEED_RHS, kmax=8):
    """Modes of the divergence of a random smooth velocity field.

    v_c = sum_{k in Z^3, 0<|k|<=kmax} |k|^-2 (a_ck cos k.x + b_ck sin k.x),
    a, b ~ N(0,1), k enumerated lexicographically over kx, ky, kz in
    [-kmax, kmax] (kx slowest), draws a_{0k} a_{1k} a_{2k} b_{0k} b_{1k} b_{2k}
    per mode.  Returns (K [m,3] int, cc [m], cs [m]) with
    div v = sum_k cc_k cos(k.x) + cs_k sin(k.x).
    """
    rng = _rng(seed)
    ks = []
    r = np.arange(-kmax, kmax + 1)
    for kx in r:
        for ky in r:
            for kz in r:
                k2 = kx * kx + ky * ky + kz * kz
                if 0 < k2 <= kmax * kmax:
                    ks.append((kx, ky, kz))
    K = np.array(ks, dtype=np.int64)
    ab = rng.standard_normal(size=(len(K), 6))
    k2 = (K * K).sum(1).astype(np.float64)
    # d/dx_c [a cos(k.x) + b sin(k.x)] = k_c (-a sin + b cos)
    cc = (K * ab[:, 3:6]).sum(1) / k2
    cs = -(K * ab[:, 0:3]).sum(1) / k2
    return K, cc, cs


def eval_fourier(K, cc, cs, x, y, z, chunk=1 << 16):
    """sum_k cc_k cos(k.x) + cs_k sin(k.x) at points (x, y, z); numpy or torch arrays.

    Uses e^{i k.x} = (e^{ix})^kx (e^{iy})^ky (e^{iz})^kz with integer powers
    tabulated per point, summed mode by mode.
    """
    try:
        import torch
        is_torch = isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_torch = False
    kmax = int(np.abs(K).max())
    if is_torch:
        import torch
        dev = x.device
        out = torch.empty(x.numel(), dtype=torch.float64, device=dev)
        n = x.numel()
        step = 1 << 22
        for s in range(0, n, step):
            sl = slice(s, min(n, s + step))
            tabs = []
            for c in (x, y, z):
                e = torch.exp(1j * c.reshape(-1)[sl].to(torch.float64))
                pw = torch.ones((2 * kmax + 1, e.numel()), dtype=torch.complex128, device=dev)
                for p in range(1, kmax + 1):
                    pw[kmax + p] = pw[kmax + p - 1] * e
                    pw[kmax - p] = pw[kmax - p + 1] * e.conj()
                tabs.append(pw)
            acc = torch.zeros(e.numel(), dtype=torch.float64, device=dev)
            for m in range(K.shape[0]):
                zz = tabs[0][K[m, 0] + kmax] * tabs[1][K[m, 1] + kmax] * tabs[2][K[m, 2] + kmax]
                acc += float(cc[m]) * zz.real + float(cs[m]) * zz.imag
            out[sl] = acc
        return out.reshape(x.shape)
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    z = np.asarray(z, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    for s in range(0, x.size, chunk):
        sl = slice(s, min(x.size, s + chunk))
        tabs = []
        for c in (x[sl], y[sl], z[sl]):
            e = np.exp(1j * c)
            pw = np.ones((2 * kmax + 1, e.size), dtype=np.complex128)
            for p in range(1, kmax + 1):
                pw[kmax + p] = pw[kmax + p - 1] * e
                pw[kmax - p] = pw[kmax - p + 1] * np.conj(e)
            tabs.append(pw)
        acc = np.zeros(e.size)
        for m in range(K.shape[0]):
            zz = tabs[0][K[m, 0] + kmax] * tabs[1][K[m, 1] + kmax] * tabs[2][K[m, 2] + kmax]
            acc += cc[m] * zz.real + cs[m] * zz.imag
        out[sl] = acc
    return out


def batch_problems(nprob=64, seed=SEED_BATCH, edges=(8, 12, 16, 20, 24), orders=(5, 7, 9)):
    """Uneven batch: per problem (edge, N, k1, k2, k3), drawn in that order."""
    rng = _rng(seed)
    out = []
    for _ in range(nprob):
        edge = int(edges[rng.integers(0, len(edges))])
        N = int(orders[rng.integers(0, len(orders))])
        k = tuple(int(v) for v in rng.integers(1, 5, size=3))
        out.append((edge, N) + k)
    return out


def sine_product(k, x, y, z, lib=np):
    """u*(x,y,z) = sin(k1 x) sin(k2 y) sin(k3 z)."""
    return lib.sin(k[0] * x) * lib.sin(k[1] * y) * lib.sin(k[2] * z)


def tgv_initial(x, y, z, lib=np, v0=1.0):
    """Taylor-Green vortex initial velocity and the pressure used as a first guess:
    u = v0 sin x cos y cos z, v = -v0 cos x sin y cos z, w = 0,
    p = (cos 2x + cos 2y)(cos 2z + 2)/16."""
    u = v0 * lib.sin(x) * lib.cos(y) * lib.cos(z)
    v = -v0 * lib.cos(x) * lib.sin(y) * lib.cos(z)
    w = 0.0 * x
    p = (lib.cos(2 * x) + lib.cos(2 * y)) * (lib.cos(2 * z) + 2.0) / 16.0
    return u, v, w, p


def tg2d_exact(x, y, z, t, nu, lib=np):
    """Exact 2-D Taylor-Green Navier-Stokes solution (extended uniformly in z):
    u = sin x cos y F, v = -cos x sin y F, w = 0, p = (cos 2x + cos 2y) F^2 / 4,
    F = exp(-2 nu t)."""
    F = math.exp(-2.0 * nu * t)
    u = lib.sin(x) * lib.cos(y) * F
    v = -lib.cos(x) * lib.sin(y) * F
    w = 0.0 * x
    p = (lib.cos(2 * x) + lib.cos(2 * y)) * F * F / 4.0
    return u, v, w, p
