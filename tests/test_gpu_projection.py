"""GPU tests of the projected pressure solve (Sec. 3: projection space of 20).

With the projection on, the Re=1600 Taylor-Green histories on 6^3 elements,
N=7, stay within the e_E,max / e_Omega,max bars of the FP64 oracle (which
solves every pressure system from the previous pressure without projection),
agree with the unprojected GPU run to the level the absolute pressure
tolerance allows, and the pressure solves need far fewer iterations once the
basis holds a few solutions.  Turning the projection off again restores the
unprojected run bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import gpu_coords, pair, torch_dev
from paper_2608_24348_gb300 import inputs, policy

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi
N, NEL, NU, DT, STEPS = 7, (6, 6, 6), 1.0 / 1600, 1e-3, 30


@pytest.fixture(scope="module")
def setup(sem):
    ctx, m, v = pair(sem, N, NEL, 0.0)
    x, y, z = m.xyz
    O = oracle.TGV(N, NEL, v, (TWO_PI,) * 3, NU, DT, tol_v=1e-6, tol_p=1e-4, abs_tol=True)
    O.set(*inputs.tgv_initial(x, y, z))
    return ctx, O.step(STEPS)


def run(sem, ctx, proj, steps=STEPS, toggle_off=False):
    torch, _ = torch_dev()
    T = sem.TGV(ctx, NU, DT, op="f64", vel=sem.opts(tol=1e-6, abs_tol=True),
                pres=sem.opts(tol=1e-4, abs_tol=True))
    if proj:
        T.set_projection(proj)
    if toggle_off:
        T.set_projection(0)
    x, y, z = gpu_coords(ctx)
    u, v, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    T.set(u.contiguous(), v.contiguous(), (w + 0 * x).contiguous(), p.contiguous())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = T.step(steps, stream=stream)
    T.close()
    return d


def test_projection_matches_oracle_and_cuts_pressure_iterations(sem, setup):
    ctx, ref = setup
    d0 = run(sem, ctx, 0)
    d1 = run(sem, ctx, 20)
    assert all(r["status"] == 0 for r in d1), [r["status"] for r in d1]
    for d in (d0, d1):
        assert policy.e_max([r["ke"] for r in d], ref[:, 1]) <= 1e-4
        assert policy.e_max([r["enstrophy"] for r in d], ref[:, 2]) <= 1e-3
    # the two GPU runs differ only through pressure solves converged to |r| <= 1e-4
    assert policy.e_max([r["ke"] for r in d1], [r["ke"] for r in d0]) <= 1e-6
    it0 = np.mean([r["iters"][0] for r in d0[10:]])
    it1 = np.mean([r["iters"][0] for r in d1[10:]])
    assert it1 <= 0.5 * it0, (it0, it1)


def test_small_basis_restarts_and_stays_accurate(sem, setup):
    ctx, ref = setup
    d = run(sem, ctx, 3)  # restarts every three steps
    assert all(r["status"] == 0 for r in d)
    assert policy.e_max([r["ke"] for r in d], ref[:, 1]) <= 1e-4
    assert policy.e_max([r["enstrophy"] for r in d], ref[:, 2]) <= 1e-3


def test_projection_off_restores_the_plain_solve(sem, setup):
    ctx, _ = setup
    a = run(sem, ctx, 0, steps=8)
    b = run(sem, ctx, 20, steps=8, toggle_off=True)
    assert [r["ke"] for r in a] == [r["ke"] for r in b]
    assert [r["iters"] for r in a] == [r["iters"] for r in b]


def test_projection_rejects_bad_sizes(sem, setup):
    ctx, _ = setup
    T = sem.TGV(ctx, NU, DT)
    for bad in (-1, 33):
        with pytest.raises(sem.SemError):
            T.set_projection(bad)
    T.close()
