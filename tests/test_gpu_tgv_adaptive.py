"""GPU parity of the stepper's step-size control (Sec. 3: adaptive steps at CFL
0.4, BDF3/EXT3 on unequal steps).

Bars: with tight solver tolerances (1e-10 relative where the steps reach CFL
0.4: at 1e-12 the pressure solve of the singular periodic Poisson problem can
meet <p,Ap> <= 0 at these steps, fixed or not) the step sizes, the CFL numbers
and the KE / enstrophy histories follow the FP64 oracle running the same rule
to 1e-8 / 1e-8 / 1e-9 / 1e-8 relative (the CFL of each step is a maximum over
nodes of the new velocity, which the two sides hold to about 1e-10); unequal
prescribed steps keep third-order convergence on the exact 2-D Taylor-Green
vortex; a fixed step changed mid-run (graph replay on both sides of the
change) matches the oracle making the same change.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import gpu_coords, pair, torch_dev
from paper_2608_24348_gb300 import inputs

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def e_max(a, ref):
    a, ref = np.asarray(a), np.asarray(ref)
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def _tight(sem, tol=1e-12):
    return dict(vel=sem.opts(tol=tol, abs_tol=False), pres=sem.opts(tol=tol, abs_tol=False))


def _ic_gpu(ctx):
    torch, _ = torch_dev()
    x, y, z = gpu_coords(ctx)
    u, v, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    return [t.contiguous() for t in (u, v, w + 0 * x, p)]


def test_cfl_controlled_steps_match_oracle(sem):
    """Re = 1600, N = 7 on 6^3 elements from dt = 1e-2 (CFL about 0.3): the
    step grows by the 10 % cap (CFL about 0.14 at the start), then settles at
    CFL 0.4 from the twelfth step; 20 steps."""
    torch, _ = torch_dev()
    N, nel, nu, dt0 = 7, (6, 6, 6), 1.0 / 1600, 1e-2
    ctx, m, v = pair(sem, N, nel, 0.0)
    T = sem.TGV(ctx, nu, dt0, **_tight(sem, 1e-10))
    T.set(*_ic_gpu(ctx))
    T.set_dt(cfl_target=0.4, dt_max=0.05)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = T.step(20, stream=stream)
    T.close()
    assert all(r["status"] == 0 for r in d), [(r["status"], r["iters"], r["dt"]) for r in d]
    O = oracle.TGV(N, nel, v, (TWO_PI,) * 3, nu, dt0, tol_v=1e-10, tol_p=1e-10, abs_tol=False)
    O.set(*inputs.tgv_initial(*m.xyz))
    O.set_dt(cfl_target=0.4, dt_max=0.05)
    ref = O.step(20)
    assert np.all(ref[:, 7] == 0)
    dts = np.array([r["dt"] for r in d])
    cfl = np.array([r["cfl"] for r in d])
    assert dts[0] == dt0 and abs(dts[1] - 1.1 * dt0) <= 1e-15   # growth capped at 10 %
    assert abs(cfl[-1] - 0.4) <= 0.01, cfl
    np.testing.assert_allclose(dts, ref[:, 8], rtol=1e-8)
    np.testing.assert_allclose(cfl, ref[:, 9], rtol=1e-8)
    np.testing.assert_allclose([r["t"] for r in d], ref[:, 0], rtol=1e-8)
    assert e_max([r["ke"] for r in d], ref[:, 1]) <= 1e-9
    assert e_max([r["enstrophy"] for r in d], ref[:, 2]) <= 1e-8


def test_unequal_steps_keep_third_order(sem):
    """Steps alternating 0.7 h and 1.3 h (with a slow drift) on the exact 2-D
    Taylor-Green vortex, nu = 0.2 to t = 1: convergence rate about 3."""
    torch, dev = torch_dev()
    nu, T_end, N, nel = 0.2, 1.0, 9, (4, 4, 1)
    ctx, _, _ = pair(sem, N, nel, 0.0, with_oracle=False)
    x, y, z = gpu_coords(ctx)
    errs = []
    for h in (0.1, 0.05, 0.025):
        T = sem.TGV(ctx, nu, h, **_tight(sem))
        for lev in (2, 1, 0):
            u, vv, w, p = inputs.tg2d_exact(x, y, z, -lev * h, nu, lib=torch)
            T.set(u.contiguous(), vv.contiguous(), (w + 0 * x).contiguous(),
                  p.contiguous() if lev == 0 else None, level=lev, step=2, t=0.0)
        t, k = 0.0, 0
        while T_end - t > 1e-12:
            dt = min(h * (0.7 if k % 2 == 0 else 1.3) * (1 + 0.1 * math.sin(t)), T_end - t)
            T.set_dt(dt)
            r = T.step(1)[0]
            assert r["status"] == 0 and abs(r["dt"] - dt) <= 1e-15
            t += dt
            k += 1
        out = [torch.empty(ctx.nL, dtype=torch.float64, device=dev) for _ in range(4)]
        T.get(*out)
        T.close()
        ue, ve, _, _ = inputs.tg2d_exact(x, y, z, T_end, nu, lib=torch)
        errs.append(max(float((out[0] - ue).abs().max()), float((out[1] - ve).abs().max())))
    rates = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert rates[0] > 2.6 and rates[1] > 2.6, (errs, rates)


def test_fixed_step_change_recaptures_the_graph(sem):
    """Ten graph-replayed steps at dt = 1e-3, then ten at 2e-3 (three steps of
    variable coefficients, then replay again): the same history as the oracle
    making the same change."""
    torch, _ = torch_dev()
    N, nel, nu = 5, (4, 4, 4), 1.0 / 1600
    ctx, m, v = pair(sem, N, nel, 0.0)
    T = sem.TGV(ctx, nu, 1e-3, **_tight(sem))
    T.set(*_ic_gpu(ctx))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = T.step(10, stream=stream)
        T.set_dt(2e-3)
        d += T.step(10, stream=stream)
    T.close()
    assert all(r["status"] == 0 for r in d), d
    O = oracle.TGV(N, nel, v, (TWO_PI,) * 3, nu, 1e-3, tol_v=1e-12, tol_p=1e-12, abs_tol=False)
    O.set(*inputs.tgv_initial(*m.xyz))
    ref = np.vstack([O.step(10), (O.set_dt(2e-3), O.step(10))[1]])
    assert [r["dt"] for r in d] == [1e-3] * 10 + [2e-3] * 10
    np.testing.assert_allclose([r["t"] for r in d], ref[:, 0], rtol=1e-13)
    assert e_max([r["ke"] for r in d], ref[:, 1]) <= 1e-10
    assert e_max([r["enstrophy"] for r in d], ref[:, 2]) <= 1e-9
    np.testing.assert_allclose([r["cfl"] for r in d], ref[:, 9], rtol=1e-8)


def test_set_dt_rejects_bad_arguments(sem):
    ctx, _, _ = pair(sem, 3, (2, 2, 2), 0.0, with_oracle=False)
    T = sem.TGV(ctx, 0.01, 1e-3)
    for bad in (dict(dt=-1.0), dict(cfl_target=float("nan")), dict(dt_max=-0.1)):
        with pytest.raises(sem.SemError):
            T.set_dt(**bad)
    T.close()
