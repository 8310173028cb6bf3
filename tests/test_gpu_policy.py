"""GPU tests of the stepper's precision policy (Sec. 2 Fig. 2; Table 2).

Every Table 2 configuration runs 20 steps of the Re=1600 Taylor-Green vortex
on 6^3 elements, N=7, with the paper's absolute solver tolerances, and its KE and
enstrophy histories are compared with the FP64 oracle by e_E,max and
e_Omega,max (Sec. 4.2, without the x100 %), bars 1e-4 and 1e-3.  A schedule
that changes rule at a step boundary reproduces the single-rule runs on both
sides of the switch, and malformed schedules are refused.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import gpu_coords, pair, torch_dev
from paper_2608_24348_gb300 import inputs, policy

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi
N, NEL, NU, DT, STEPS = 7, (6, 6, 6), 1.0 / 1600, 1e-3, 20


@pytest.fixture(scope="module")
def setup(sem):
    ctx, m, v = pair(sem, N, NEL, 0.0)
    x, y, z = m.xyz
    O = oracle.TGV(N, NEL, v, (TWO_PI,) * 3, NU, DT, tol_v=1e-6, tol_p=1e-4, abs_tol=True)
    O.set(*inputs.tgv_initial(x, y, z))
    ref = O.step(STEPS)
    assert np.all(ref[:, 7] == 0)
    return ctx, ref


def run(sem, ctx, rules, steps=STEPS):
    torch, _ = torch_dev()
    T = sem.TGV(ctx, NU, DT, op="f64", vel=sem.opts(tol=1e-6, abs_tol=True, maxit=3000),
                pres=sem.opts(tol=1e-4, abs_tol=True, maxit=3000))
    T.set_policy(rules)
    x, y, z = gpu_coords(ctx)
    u, v, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    T.set(u.contiguous(), v.contiguous(), (w + 0 * x).contiguous(), p.contiguous())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = T.step(steps, stream=stream)
    T.close()
    return d


@pytest.mark.parametrize("name", list(policy.TABLE2))
def test_table2_configuration_matches_oracle(sem, setup, name):
    ctx, ref = setup
    d = run(sem, ctx, [policy.rule(name)])
    assert all(r["status"] == 0 for r in d), (name, [r["status"] for r in d])
    np.testing.assert_allclose([r["t"] for r in d], ref[:, 0], rtol=1e-12)
    eE = policy.e_max([r["ke"] for r in d], ref[:, 1])
    eO = policy.e_max([r["enstrophy"] for r in d], ref[:, 2])
    assert eE <= 1e-4 and eO <= 1e-3, (name, eE, eO)
    if name == "A-0":  # FP64 throughout: the oracle's histories to solver tolerance
        assert eE <= 1e-8 and eO <= 1e-7, (eE, eO)


def test_schedule_switches_at_step_boundary(sem, setup):
    ctx, _ = setup
    a0 = run(sem, ctx, [policy.rule("A-0")])
    b0 = run(sem, ctx, [policy.rule("B-0")])
    sw = run(sem, ctx, [policy.rule("A-0"), policy.rule("B-0", first_step=11)])
    ke = lambda d: np.array([r["ke"] for r in d])
    assert np.array_equal(ke(sw)[:10], ke(a0)[:10])  # identical before the switch
    assert not np.array_equal(ke(sw)[10:], ke(a0)[10:])  # B-0 numerics after it
    assert policy.e_max(ke(sw), ke(a0)) <= 1e-4
    assert policy.e_max(ke(b0), ke(a0)) <= 1e-4
    # an empty schedule restores the constructor's precisions (here FP64)
    assert np.array_equal(ke(run(sem, ctx, [])), ke(a0))


def test_storage_rounding_is_fp32_representable(sem, setup):
    torch, dev = torch_dev()
    ctx, _ = setup
    T = sem.TGV(ctx, NU, DT, op="f64", vel=sem.opts(tol=1e-6, abs_tol=True),
                pres=sem.opts(tol=1e-4, abs_tol=True))
    T.set_policy([policy.rule("B-1")])
    x, y, z = gpu_coords(ctx)
    u, v, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    T.set(u.contiguous(), v.contiguous(), (w + 0 * x).contiguous(), p.contiguous())
    T.step(3)
    out = [torch.empty(ctx.nL, dtype=torch.float64, device=dev) for _ in range(4)]
    T.get(*out)
    for a in out:  # every stored value is an FP32 number
        assert torch.equal(a, a.float().double())
    T.close()


def test_malformed_schedules_are_refused(sem, setup):
    ctx, _ = setup
    T = sem.TGV(ctx, NU, DT)
    with pytest.raises(sem.SemError):
        T.set_policy([policy.rule("A-0", 5), policy.rule("A-1", 2)])  # unsorted
    with pytest.raises(sem.SemError):
        T.set_policy([dict(policy.TABLE2["A-0"], storage="bf16_tc")])  # no 16-bit storage
    with pytest.raises(sem.SemError):
        T.set_policy([policy.rule("A-0")] * 9)  # more than SEM_TGV_MAX_RULES
    T.close()


def test_fp32_storage_matches_the_oracle_with_fp32_storage(sem):
    """B-1 (FP64 compute, rp = fp32 storage) against the oracle run with the same
    FP32 rounding of the stored state: the histories agree to FP64 round-off,
    while the FP64-storage oracle differs by the FP32 rounding of the state."""
    torch, _ = torch_dev()
    n, nel, steps = 5, (3, 3, 3), 6
    ctx, m, v = pair(sem, n, nel, 0.0)
    T = sem.TGV(ctx, NU, DT, op="f64", vel=sem.opts(tol=1e-12), pres=sem.opts(tol=1e-12))
    T.set_policy([policy.rule("B-1")])
    x, y, z = gpu_coords(ctx)
    u, vv, w, p = inputs.tgv_initial(x, y, z, lib=torch)
    T.set(u.contiguous(), vv.contiguous(), (w + 0 * x).contiguous(), p.contiguous())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = T.step(steps, stream=stream)
    T.close()
    assert all(r["status"] == 0 for r in d)
    xo, yo, zo = m.xyz
    ref = {}
    for store32 in (True, False):
        O = oracle.TGV(n, nel, v, (TWO_PI,) * 3, NU, DT, tol_v=1e-12, tol_p=1e-12, abs_tol=False)
        O.set_storage(store32)
        O.set(*inputs.tgv_initial(xo, yo, zo))
        ref[store32] = O.step(steps)
    for col, key in ((1, "ke"), (2, "enstrophy")):
        h = [r[key] for r in d]
        e32 = policy.e_max(h, ref[True][:, col])
        e64 = policy.e_max(h, ref[False][:, col])
        assert e32 <= 2e-11 and e64 >= 5e-10, (key, e32, e64)
