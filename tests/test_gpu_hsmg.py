"""GPU parity of the pressure solver: flexible GMRES with the hybrid Schwarz
multigrid preconditioner (Sec. 1; Sec. 3 solver settings).

Bars: one V-cycle in FP64 with a tight coarse solve matches the oracle's to
1e-10 relative (the FP32 V-cycle to 1e-5); unpreconditioned GMRES reaches the
oracle's minimal residual after k steps to 1e-9; preconditioned GMRES solutions
match the oracle's to 1e-8 with iteration counts within 2; at full size (32^3,
N=7) the pressure Poisson problem converges to 1e-10 in a small fraction of
Jacobi-PCG's iterations, with the solution within 1e-8 of the PCG solution;
the stepper with the GMRES pressure solver follows the oracle stepper.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import fourier_rhs, gpu_coords, pair, torch_dev
from paper_2608_24348_gb300 import inputs

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def _rhs(sem, ctx, m, seed=3):
    """A continuous assembled right-hand side on both sides: dssum of seeded local values."""
    torch, dev = torch_dev()
    f = np.random.default_rng(seed).standard_normal(ctx.nL)
    bo = m.dssum(f)
    bg = torch.from_numpy(bo).to(dev)
    return bg, bo


@pytest.mark.parametrize("N,nel,periodic,orders,h2", [
    (5, (4, 3, 3), (1, 1, 1), [5, 3, 1], 0.0),
    (7, (3, 3, 2), (1, 1, 1), [7, 3, 1], 0.0),
    (4, (3, 2, 3), (0, 1, 0), [4, 2, 1], 2.5),
])
def test_vcycle_matches_oracle(sem, N, nel, periodic, orders, h2):
    torch, dev = torch_dev()
    ctx, m, v = pair(sem, N, nel, 0.1, periodic=periodic)
    bg, bo = _rhs(sem, ctx, m)
    ref = oracle.HSMG(orders, nel, v, periodic=periodic, h2=h2, ctol=1e-13, cmaxit=5000).apply(bo)
    for dt, bar in (("f64", 1e-10), ("f32", 1e-5)):
        H = sem.HSMG(ctx, orders, h2=h2, dtype=dt, coarse_tol=1e-13, coarse_maxit=5000)
        z = torch.empty_like(bg)
        H.apply(bg, z)
        torch.cuda.synchronize()
        assert rel(z.cpu().numpy(), ref) <= bar, (dt, rel(z.cpu().numpy(), ref))
        H.close()


def test_gmres_without_preconditioner_is_the_minimal_residual(sem):
    """k unrestarted steps: the GPU's true residual equals the oracle GMRES's (the
    minimal residual over the Krylov space, pinned in the oracle's tests)."""
    torch, dev = torch_dev()
    N, nel, h2 = 3, (3, 2, 3), 1.5
    ctx, m, v = pair(sem, N, nel, 0.1)
    bg, bo = _rhs(sem, ctx, m, seed=8)
    H = sem.HSMG(ctx, [3, 1], h2=h2, dtype="f64")
    for k in (1, 4, 9):
        x = torch.zeros_like(bg)
        info = H.gmres(bg, x, restart=20, precond=False, tol=1e-30, maxit=k)
        xo, st, io = oracle.fgmres(bo, mesh=m, h1=1.0, h2=h2, tol=1e-30, m=20, maxit=k)
        assert info["iters"] == k == io["iters"]
        assert abs(info["rnorm"] - io["rnorm"]) <= 1e-9 * io["bnorm"], (k, info, io)
        assert rel(x.cpu().numpy(), xo) <= 1e-8
    H.close()


@pytest.mark.parametrize("N,nel,orders,dt", [(5, (4, 4, 3), [5, 3, 1], "f32"),
                                             (7, (3, 3, 3), [7, 3, 1], "f64")])
def test_preconditioned_gmres_matches_oracle(sem, N, nel, orders, dt):
    torch, dev = torch_dev()
    ctx, m, v = pair(sem, N, nel, 0.1)
    bg, bo = _rhs(sem, ctx, m, seed=4)
    H = sem.HSMG(ctx, orders, dtype=dt, coarse_tol=1e-2)
    x = torch.zeros_like(bg)
    info = H.gmres(bg, x, restart=30, tol=1e-10)
    xo, st, io = oracle.fgmres(bo, hsmg=oracle.HSMG(orders, nel, v, ctol=1e-2), tol=1e-10, m=30,
                               maxit=500)
    assert info["status"] == 0 and st == 0
    assert abs(info["iters"] - io["iters"]) <= 2, (info, io)
    assert rel(x.cpu().numpy(), xo) <= 1e-8
    r, bn = m.residual(bo, x.cpu().numpy())
    assert r <= 1.5e-10 * bn
    H.close()


def test_gmres_status_and_restarts(sem):
    torch, dev = torch_dev()
    ctx, m, v = pair(sem, 5, (3, 3, 3), 0.1)
    bg, bo = _rhs(sem, ctx, m, seed=6)
    H = sem.HSMG(ctx, [5, 3, 1], dtype="f32")
    x = torch.zeros_like(bg)
    info = H.gmres(bg, x, restart=3, tol=1e-12, maxit=4)
    assert info["status"] == sem.ERR_NOT_CONVERGED and info["iters"] == 4 and info["outer_iters"] >= 1
    assert 0 < info["rnorm"] < info["bnorm"]
    x.zero_()
    info = H.gmres(bg, x, restart=4, tol=1e-9, maxit=400)    # restarted to convergence
    assert info["status"] == 0 and info["outer_iters"] >= 1
    z = torch.zeros_like(bg)
    x.zero_()
    info = H.gmres(z, x, tol=1e-9)                             # zero right-hand side and guess
    assert info["status"] == 0 and info["iters"] == 0
    with pytest.raises(sem.SemError):
        H.gmres(bg, x, restart=0)
    H.close()


def test_full_size_pressure_poisson(sem):
    """32^3, N=7 undeformed (the Taylor-Green box), Fourier right-hand side: GMRES +
    HSMG to 1e-10 in at most 40 iterations, against Jacobi-PCG's hundreds."""
    torch, dev = torch_dev()
    ctx, _, _ = pair(sem, 7, (32, 32, 32), 0.0, with_oracle=False)
    bg, _ = fourier_rhs(ctx, None)
    H = sem.HSMG(ctx, [7, 3, 1], dtype="f32")
    x = torch.zeros_like(bg)
    torch.cuda.synchronize()
    info = H.gmres(bg, x, restart=30, tol=1e-10)
    xp = torch.zeros_like(bg)
    ip = ctx.pcg_solve(bg, xp, tol=1e-10)
    assert info["status"] == 0 and ip["status"] == 0
    assert info["iters"] <= 40 and info["iters"] * 10 <= ip["iters"], (info, ip)
    assert info["rnorm"] <= 1e-10 * info["bnorm"]  # true residual, native FP64 operator
    d = (x - xp).abs().max().item() / xp.abs().max().item()
    assert d <= 1e-8, d
    H.close()


def test_stepper_with_gmres_pressure_matches_oracle(sem):
    """20 Taylor-Green steps (6^3, N=7, Re=1600) with the GMRES + HSMG pressure solve
    and tight tolerances follow the oracle stepper (Jacobi-PCG pressure: the
    pressure is the same to the tolerance), with few GMRES iterations per step."""
    torch, dev = torch_dev()
    N, nel, nu, dt = 7, (6, 6, 6), 1.0 / 1600, 1e-3
    ctx, m, v = pair(sem, N, nel, 0.0)
    T = sem.TGV(ctx, nu, dt, vel=sem.opts(tol=1e-12, abs_tol=False), pres=sem.opts(tol=1e-10, abs_tol=False))
    T.set_pressure_solver("gmres_hsmg", restart=30, vcycle="f32")
    x, y, z = gpu_coords(ctx)
    u, vv, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    T.set(u.contiguous(), vv.contiguous(), (w + 0 * x).contiguous(), p.contiguous())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = T.step(20, stream=stream)
    T.close()
    assert all(r["status"] == 0 for r in d), d
    O = oracle.TGV(N, nel, v, (TWO_PI,) * 3, nu, dt, tol_v=1e-12, tol_p=1e-10, abs_tol=False)
    O.set(*inputs.tgv_initial(*m.xyz))
    ref = O.step(20)
    assert rel([r["ke"] for r in d], ref[:, 1]) <= 1e-9
    assert rel([r["enstrophy"] for r in d], ref[:, 2]) <= 1e-8
    its = [r["iters"][0] for r in d]
    assert max(its[3:]) <= 25 and np.mean(its) < ref[:, 3].mean() / 3, (its, ref[:, 3])


def test_stepper_switches_pressure_solvers(sem):
    """Jacobi-PCG (graph replay), then GMRES + HSMG (direct launches, FP64 V-cycle),
    then Jacobi-PCG again, 5 steps each with tight tolerances: the history follows
    the oracle stepper throughout; bad arguments are rejected."""
    torch, dev = torch_dev()
    N, nel, nu, dt = 5, (4, 4, 4), 1.0 / 1600, 2e-3
    ctx, m, v = pair(sem, N, nel, 0.0)
    T = sem.TGV(ctx, nu, dt, vel=sem.opts(tol=1e-12, abs_tol=False), pres=sem.opts(tol=1e-10, abs_tol=False))
    x, y, z = gpu_coords(ctx)
    u, vv, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    T.set(u.contiguous(), vv.contiguous(), (w + 0 * x).contiguous(), p.contiguous())
    stream = torch.cuda.Stream()
    d = []
    with torch.cuda.stream(stream):
        d += T.step(5, stream=stream)
        T.set_pressure_solver("gmres_hsmg", restart=20, vcycle="f64")
        d += T.step(5, stream=stream)
        T.set_pressure_solver("pcg")
        d += T.step(5, stream=stream)
    for bad in (dict(restart=0), dict(restart=65), dict(vcycle="bf16_tc")):
        with pytest.raises(sem.SemError):
            T.set_pressure_solver("gmres_hsmg", **bad)
    T.close()
    assert all(r["status"] == 0 for r in d), d
    O = oracle.TGV(N, nel, v, (TWO_PI,) * 3, nu, dt, tol_v=1e-12, tol_p=1e-10, abs_tol=False)
    O.set(*inputs.tgv_initial(*m.xyz))
    ref = O.step(15)
    assert rel([r["ke"] for r in d], ref[:, 1]) <= 1e-9
    assert rel([r["enstrophy"] for r in d], ref[:, 2]) <= 1e-8
    its = [r["iters"][0] for r in d]
    assert max(its[5:10]) < min(its[10:]), its   # GMRES + HSMG against Jacobi-PCG iterations
