"""The block-floating-point FP64-accurate operator (sem_ax SEM_F64 for even
N+1 <= 12: its candidates 3 and 4 (direct loads; scalar or paired f32x2
instructions), 5 and 6 (u staged by bulk copies), 8 (staged, one element per
block, the default) and 9, 10 (other register budgets)) against the FP64
oracle.

Bar: max|gpu - ref| / max|ref| <= 1e-12, the FP64 operator's bar.  Cases span
every even N+1 the kernel serves, several element groups and a ragged tail,
both (h1, h2) pairs, deformed meshes, continuous and discontinuous inputs,
elements whose scales differ by up to 2^200 (the per-element exponent), an
all-zero element and a smooth field (the operator's cancellation case).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_24348_gb300 import inputs

pytestmark = pytest.mark.gpu

TWO_PI = 2 * math.pi
BFP = (3, 4, 5, 6, 8, 9, 10)


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def make(sem, N, nel, perturb, periodic=(1, 1, 1)):
    v = inputs.box_vertices(nel, (TWO_PI,) * 3, perturb=perturb)
    ctx = sem.Ctx(N, nel, (TWO_PI,) * 3, periodic, vertices=v)
    return ctx, oracle.Mesh(N, nel, v, periodic), v


def run(sem, ctx, u, h1, h2):
    """Every candidate's result; the two are bit-identical (same roundings)."""
    torch, dev = torch_dev()
    ud = torch.from_numpy(np.ascontiguousarray(u)).to(dev)
    outs = []
    for v in BFP:
        wd = torch.empty_like(ud)
        sem.set_ax_variant(ctx.N, "f64", v)
        try:
            ctx.ax(ud, wd, h1, h2, "f64")
            torch.cuda.synchronize()
        finally:
            sem.set_ax_variant(ctx.N, "f64", -1)
        outs.append(wd.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    return outs[0]


@pytest.mark.parametrize("N,nel,perturb", [(1, (3, 2, 5), 0.1), (3, (2, 3, 2), 0.15),
                                           (5, (4, 4, 3), 0.1), (7, (3, 5, 2), 0.1),
                                           (9, (2, 2, 3), 0.1), (11, (2, 1, 2), 0.1)])
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.01, 1000.0)])
def test_bfp_matches_oracle(sem, N, nel, perturb, h1, h2):
    ctx, m, _ = make(sem, N, nel, perturb)
    for u in (inputs.local_uniform_field(ctx.nL, seed=inputs.SEED_FIELD),
              inputs.unique_uniform_field(N, nel, seed=inputs.SEED_FIELD)):
        ref = m.ax(u, h1, h2)
        err = rel_err(run(sem, ctx, u, h1, h2), ref)
        print(f"N={N} h1={h1} h2={h2}: {err:.3e}")
        assert err <= 1e-12, err


def test_bfp_element_scales_and_zero_element(sem):
    """Element e is scaled by 2^(40 (e mod 11) - 200); element 3 is zero.  Each
    element's result meets the bar relative to its own largest value."""
    N, nel = 7, (4, 3, 2)
    ctx, m, _ = make(sem, N, nel, 0.1)
    n3 = (N + 1) ** 3
    u = inputs.local_uniform_field(ctx.nL, seed=21).reshape(ctx.E, n3)
    u *= np.ldexp(1.0, 40 * (np.arange(ctx.E) % 11) - 200)[:, None]
    u[3] = 0.0
    u = u.reshape(-1)
    ref = m.ax(u, 0.5, 7.0).reshape(ctx.E, n3)
    got = run(sem, ctx, u, 0.5, 7.0).reshape(ctx.E, n3)
    assert np.all(got[3] == 0.0)
    for e in range(ctx.E):
        if e != 3:
            assert rel_err(got[e], ref[e]) <= 1e-12, e


def test_bfp_smooth_field_cancellation(sem):
    """u = sin x sin y sin z with h2 = 0: A u is much smaller than the terms it
    sums.  The error is measured against the operator's scale on inputs of the
    same magnitude (max |A r| for r uniform in [-1, 1] per node), the scale
    that bounds an FP64 evaluation's rounding too."""
    N, nel = 7, (4, 4, 4)
    ctx, m, _ = make(sem, N, nel, 0.1)
    x, y, z = m.xyz
    u = np.sin(x) * np.sin(y) * np.sin(z)
    ref = m.ax(u, 1.0, 0.0)
    scale = np.abs(m.ax(inputs.local_uniform_field(ctx.nL, seed=5), 1.0, 0.0)).max()
    got = run(sem, ctx, u, 1.0, 0.0)
    err = np.abs(got - ref).max() / scale
    print(f"smooth: {err:.3e} (max|Au| / scale = {np.abs(ref).max() / scale:.3e}, "
          f"relative to max|Au|: {rel_err(got, ref):.3e})")
    assert err <= 1e-12, err


def test_bfp_full_size_sampled(sem):
    """32^3 elements, N=7, deformed: 48 sampled elements against the oracle."""
    torch, dev = torch_dev()
    N, nel = 7, (32, 32, 32)
    v = inputs.box_vertices(nel, (TWO_PI,) * 3, perturb=0.1)
    ctx = sem.Ctx(N, nel, (TWO_PI,) * 3, (1, 1, 1), vertices=v)
    u = inputs.unique_uniform_field(N, nel, seed=inputs.SEED_FIELD)
    w = run(sem, ctx, u, 0.01, 1000.0).reshape(ctx.E, -1)
    u = u.reshape(ctx.E, -1)
    rng = np.random.default_rng(11)
    err = 0.0
    for e in [0, ctx.E - 1] + list(rng.choice(ctx.E, 46, replace=False)):
        ex, ey, ez = e % 32, (e // 32) % 32, e // 1024
        me = oracle.Mesh(N, (1, 1, 1), v[ez:ez + 2, ey:ey + 2, ex:ex + 2, :], (0, 0, 0))
        ref = me.ax(u[e], 0.01, 1000.0)
        err = max(err, np.abs(w[e] - ref).max() / np.abs(ref).max())
    print(f"full size sampled: {err:.3e}")
    assert err <= 1e-12, err
