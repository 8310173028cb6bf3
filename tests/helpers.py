"""Shared test helpers: build matching GPU / oracle problems from seeded inputs."""
import math

import numpy as np

import oracle
from paper_2608_24348_gb300 import inputs

TWO_PI = 2 * math.pi


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def pair(sem, N, nel, perturb=0.0, periodic=(1, 1, 1), L=(TWO_PI,) * 3, with_oracle=True):
    """(libsem context, oracle mesh, vertices) on the same seeded mesh."""
    v = inputs.box_vertices(nel, L, perturb=perturb)
    ctx = sem.Ctx(N, nel, L, periodic, vertices=v)
    m = oracle.Mesh(N, nel, v, periodic) if with_oracle else None
    return ctx, m, v


def gpu_coords(ctx):
    torch, dev = torch_dev()
    xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.coords(xyz)
    return xyz.view(3, -1)


def gpu_weak_rhs(ctx, f):
    """b = dssum(B f) on the GPU (sem_ax with h1 = 0, h2 = 1, then sem_dssum)."""
    torch, _ = torch_dev()
    b = torch.empty_like(f)
    ctx.ax(f.contiguous(), b, 0.0, 1.0, "f64")
    ctx.dssum(b, "f64")
    return b


def sine_rhs(sem_ctx, m, k=(1, 1, 1)):
    """Manufactured u* = prod sin(k_i x_i), f = |k|^2 u*: (b_gpu, b_oracle, u*_oracle)."""
    torch, _ = torch_dev()
    x, y, z = gpu_coords(sem_ctx)
    kk = float(sum(v * v for v in k))
    fg = kk * inputs.sine_product(k, x, y, z, lib=torch)
    bg = gpu_weak_rhs(sem_ctx, fg)
    bo = us = None
    if m is not None:
        us = inputs.sine_product(k, *m.xyz)
        bo = m.dssum(m.B * kk * us)
    return bg, bo, us


def fourier_rhs(sem_ctx, m):
    """Pressure-Poisson workload: f = div v of a seeded random smooth field."""
    K, cc, cs = inputs.fourier_div_modes()
    x, y, z = gpu_coords(sem_ctx)
    fg = inputs.eval_fourier(K, cc, cs, x, y, z)
    bg = gpu_weak_rhs(sem_ctx, fg)
    bo = None
    if m is not None:
        fo = oracle.fourier(K, cc, cs, *m.xyz)
        bo = m.dssum(m.B * fo)
    return bg, bo


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
