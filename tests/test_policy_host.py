"""Host-side checks of the precision-policy table and error metrics (no GPU).

The 13 configurations must be the ones Table 2 lists (Sec. 4): Group A with
rp = fp64 storage, one block lowered to fp32 in A-2..A-4; Group B with rp =
fp32 storage, one block raised to fp64 in B-2..B-4 and one fp16 kernel
override in B-5..B-7 (adv_dealias in the SEM block, ax_helm in the velocity
and the pressure block).  The metrics follow Sec. 4.2: e_max takes the largest
pointwise difference over the largest reference value, e_peak the difference of
the two maxima over the largest reference value.
"""
import ctypes
import os
import re

import pytest

from paper_2608_24348_gb300 import policy, sem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BLOCKS = ("sem", "vel", "pres")


def test_table2_has_the_papers_thirteen_configurations():
    assert list(policy.TABLE2) == [f"A-{k}" for k in range(5)] + [f"B-{k}" for k in range(8)]
    for name, r in policy.TABLE2.items():
        assert r["storage"] == ("f64" if name.startswith("A") else "f32")


@pytest.mark.parametrize("name,lowered", [("A-1", BLOCKS), ("A-2", ("sem",)), ("A-3", ("vel",)),
                                          ("A-4", ("pres",)), ("A-0", ())])
def test_group_a_lowers_the_named_blocks_to_fp32(name, lowered):
    r = policy.TABLE2[name]
    for b in BLOCKS:
        assert r[b] == ("f32" if b in lowered else "f64"), (name, b)


@pytest.mark.parametrize("name,raised", [("B-1", BLOCKS), ("B-2", ("sem",)), ("B-3", ("vel",)),
                                         ("B-4", ("pres",)), ("B-0", ())])
def test_group_b_raises_the_named_blocks_to_fp64(name, raised):
    r = policy.TABLE2[name]
    for b in BLOCKS:
        assert r[b] == ("f64" if b in raised else "f32"), (name, b)


@pytest.mark.parametrize("name,block", [("B-5", "sem"), ("B-6", "vel"), ("B-7", "pres")])
def test_group_b_fp16_kernel_overrides(name, block):
    r = policy.TABLE2[name]
    for b in BLOCKS:
        assert r[b] == ("f16_tc" if b == block else "f32"), (name, b)


def test_rule_adds_the_first_step_and_copies():
    r = policy.rule("B-6", first_step=101)
    assert r["first_step"] == 101 and r["vel"] == "f16_tc"
    r["vel"] = "f64"
    assert policy.TABLE2["B-6"]["vel"] == "f16_tc"


def test_error_metrics_on_a_worked_example():
    ref = [1.0, 4.0, 2.0]
    mxp = [1.2, 3.5, 2.0]
    # largest pointwise difference 0.5 (at the second sample) over max |ref| = 4
    assert policy.e_max(mxp, ref) == pytest.approx(0.125)
    # maxima 3.5 and 4.0 (same sample here)
    assert policy.e_peak(mxp, ref) == pytest.approx(0.125)
    # peaks at different samples: e_peak compares the maxima, not the samples
    late = [1.0, 2.0, 4.4]
    assert policy.e_peak(late, ref) == pytest.approx(0.1)
    assert policy.e_max(late, ref) == pytest.approx(0.6)
    assert policy.e_max(ref, ref) == 0.0


def test_policy_struct_matches_the_c_header():
    text = open(os.path.join(ROOT, "include", "sem.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} sem_tgv_policy;", text).group(1)
    fields = re.findall(r"\b(\w+)\s*[,;]", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert fields == [f for f, _ in sem.TgvPolicy._fields_]
    assert ctypes.sizeof(sem.TgvPolicy) == 5 * ctypes.sizeof(ctypes.c_int)
    m = re.search(r"#define SEM_TGV_MAX_RULES (\d+)", text)
    assert m and int(m.group(1)) == 8


def test_peak_is_the_vertex_of_the_parabola_through_the_top_samples():
    t = [0.1 * i for i in range(20)]
    # an exact parabola: the vertex is recovered between samples
    tp, yp = policy.peak(t, [3 - (x - 0.537) ** 2 for x in t])
    assert tp == pytest.approx(0.537, abs=1e-12) and yp == pytest.approx(3.0, abs=1e-12)
    # a smooth non-parabolic peak: error of the three-point vertex is O(dt^3) in time
    import math
    tp, yp = policy.peak(t, [math.exp(-(x - 1.234) ** 2) for x in t])
    assert abs(tp - 1.234) < 2e-3 and abs(yp - 1.0) < 1e-4
    # a maximum at the end of the record stays the last sample
    assert policy.peak(t, t) == (pytest.approx(1.9), pytest.approx(1.9))


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = 0.0

    def record(self, stream=None):
        import time
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return 1000.0 * (other.t - self.t)


class _FakeStream:
    def synchronize(self):
        pass


class _FakeMeter:
    """EnergyMeter stand-in: 250 J per measured run."""
    reason = None

    def __init__(self, device=0):
        self.j = None

    def start(self):
        self.j = None

    def stop(self):
        self.j = 250.0
        return self.j

    def close(self):
        pass


class _FakeCtx:
    def __init__(self, N, nel, L, periodic):
        self.nL = 8

    def coords(self, xyz):
        xyz.zero_()


def _fake_tgv_class(histories, speed=None):
    """TGV stand-in whose KE / enstrophy follow histories[config](t); with
    set_dt(cfl_target=...) its steps follow the CFL rule for a CFL number of
    speed[config] * dt."""
    class FakeTGV:
        pressure_kinds = []

        def __init__(self, ctx, nu, dt, op, vel, pres):
            self.dt, self.n, self.cfg, self.t, self.target, self.dt_max = dt, 0, None, 0.0, 0.0, 0.0

        def set_dt(self, dt=0.0, cfl_target=0.0, dt_max=0.0):
            self.target, self.dt_max = cfl_target, dt_max

        def set_pressure_solver(self, kind="gmres_hsmg", restart=30, vcycle="f32"):
            assert kind in ("pcg", "gmres_hsmg")
            FakeTGV.pressure_kinds.append(kind)

        def set_policy(self, rules):
            self.cfg = [k for k, v in policy.TABLE2.items() if all(rules[0][b] == v[b] for b in v)][0]

        def set_projection(self, n):
            pass

        def set(self, *fields):
            pass

        def energy(self):
            return histories[self.cfg](0.0)[:2]

        def step(self, n, stream=None):
            out = []
            for _ in range(n):
                self.n += 1
                if self.target:
                    self.t += self.dt
                else:
                    self.t = self.n * self.dt
                t = self.t
                cfl = (speed or {}).get(self.cfg, 10.0) * self.dt
                ke, en, status = histories[self.cfg](t)
                out.append(dict(t=t, ke=ke, enstrophy=en, iters=[3, 2, 2, 2], status=status,
                                dt=self.dt, cfl=cfl))
                if self.target:
                    f = min(1.1, max(0.5, self.target / cfl))
                    self.dt = self.dt * f
                    if self.dt_max:
                        self.dt = min(self.dt, self.dt_max)
            return out

        def close(self):
            pass
    return FakeTGV


def test_long_run_bookkeeping_without_a_gpu(monkeypatch):
    """Chunked stepping, the stop conditions, the enstrophy peak, the dissipation
    from the KE history and the errors against A-0, on a stepper stand-in with
    closed-form histories."""
    import math

    import torch

    def a0(t):  # KE decays at rate 2 nu Omega with Omega = 1 + exp(-(t-3)^2) (nu = 1/2)
        ke = 0.125 - (t + math.sqrt(math.pi) / 2 * (math.erf(t - 3) + math.erf(3)))
        return ke + 10.0, 1.0 + math.exp(-(t - 3) ** 2), 0

    def a1(t):  # 1e-6 relative off A-0
        ke, en, _ = a0(t)
        return ke * (1 + 1e-6), en * (1 + 1e-6), 0

    def b0(t):  # diverges at t = 2
        ke, en, _ = a0(t)
        return (float("nan"), en, 0) if t >= 2.0 else (ke, en, 0)

    def b5(t):  # a solve fails at t = 1
        ke, en, _ = a0(t)
        return ke, en, (-4 if t >= 1.0 else 0)

    monkeypatch.setattr(sem, "Ctx", _FakeCtx)
    monkeypatch.setattr(sem, "TGV", _fake_tgv_class({"A-0": a0, "A-1": a1, "B-0": b0, "B-5": b5}))
    monkeypatch.setattr(sem, "opts", lambda **kw: kw)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: __import__("contextlib").nullcontext())
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **kw: real_empty(*a, **kw))
    rows = policy.long_run(["A-0", "A-1", "B-0", "B-5"], nel=2, N=3, re=2.0, dt=0.01, t_end=6.0,
                           projection=4, chunk=70, every=50)
    r = {row["config"]: row for row in rows}
    assert r["A-0"]["steps"] == 600 and r["A-0"]["stopped"] is None
    assert r["A-0"]["t_peak"] == pytest.approx(3.0, abs=1e-6)
    assert r["A-0"]["enstrophy_peak"] == pytest.approx(2.0, abs=1e-5)
    assert r["A-0"]["eps_peak"] == pytest.approx(2.0, abs=1e-5)          # 2 nu Omega, nu = 1/2
    assert r["A-0"]["eps_ke_at_peak"] == pytest.approx(2.0, rel=1e-3)    # -dKE/dt of the history
    assert len(r["A-0"]["series"]) == 12 and r["A-0"]["series"][0][0] == pytest.approx(0.5)
    assert r["A-0"]["e_E_max"] == 0.0 and r["A-1"]["e_Omega_max"] == pytest.approx(1e-6, rel=1e-3)
    # B-0 stops in the chunk where KE turned non-finite, B-5 in the one with the failed solve
    assert r["B-0"]["stopped"] == "non-finite KE or enstrophy" and 200 <= r["B-0"]["steps"] < 270
    assert r["B-5"]["stopped"] == "solve status -4" and 100 <= r["B-5"]["steps"] < 170
    assert r["B-5"]["e_Omega_max"] == 0.0  # errors over the steps both runs reached
    assert "ke" not in r["A-0"] and all(row["pres_iters"] == 3.0 for row in rows)


def test_replay_bookkeeping_without_a_gpu(monkeypatch):
    """Table 2 replay on a stepper stand-in: A-0 is prepended as the reference,
    the timed steps exclude the start-up ones, iteration means and the worst
    status are reported, and a configuration whose start-up solve fails keeps
    only those steps and no timing."""
    import math

    import torch

    def a0(t):
        return 0.125 * math.exp(-t), 0.375 * (1 + t), 0

    def a4(t):
        ke, en, _ = a0(t)
        return ke * (1 + 2e-7), en * (1 - 3e-7), 0

    def b7(t):  # the second start-up step fails to converge
        ke, en, _ = a0(t)
        return ke, en, (-5 if t >= 0.02 - 1e-12 else 0)

    monkeypatch.setattr(sem, "Ctx", _FakeCtx)
    monkeypatch.setattr(sem, "TGV", _fake_tgv_class({"A-0": a0, "A-4": a4, "B-7": b7}))
    monkeypatch.setattr(sem, "opts", lambda **kw: kw)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: __import__("contextlib").nullcontext())
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **kw: real_empty(*a, **kw))
    rows = policy.replay(["A-4", "B-7"], nel=2, N=3, dt=0.01, steps=40, warm=3, projection=4)
    r = {row["config"]: row for row in rows}
    assert [row["config"] for row in rows] == ["A-0", "A-4", "B-7"]
    assert r["A-0"]["steps"] == 40 and r["A-0"]["ms_per_step"] >= 0 and r["A-0"]["status"] == 0
    assert r["A-0"]["pres_iters"] == 3.0 and r["A-0"]["vel_iters"] == 2.0
    assert r["A-4"]["e_E_max"] == pytest.approx(2e-7, rel=1e-3)
    assert r["A-4"]["e_Omega_max"] == pytest.approx(3e-7, rel=1e-3)
    assert r["B-7"]["steps"] == 3 and r["B-7"]["status"] == -5 and math.isnan(r["B-7"]["ms_per_step"])
    assert r["B-7"]["e_E_max"] == 0.0


def _patch_gpu(monkeypatch, histories, speed=None):
    import torch

    from paper_2608_24348_gb300 import energy
    monkeypatch.setattr(sem, "Ctx", _FakeCtx)
    monkeypatch.setattr(sem, "TGV", _fake_tgv_class(histories, speed))
    monkeypatch.setattr(sem, "opts", lambda **kw: kw)
    monkeypatch.setattr(energy, "EnergyMeter", _FakeMeter)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: __import__("contextlib").nullcontext())
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **kw: real_empty(*a, **kw))


def test_cfl_controlled_long_run_without_a_gpu(monkeypatch):
    """CFL-controlled long run on the stand-in: the run ends at the first step
    reaching t_end, the step settles where speed * dt = 0.4 (growth capped at
    10 %), energy-to-solution comes from the meter, and the errors compare the
    histories at A-0's times although the two runs step differently."""
    import math

    def a0(t):
        return 0.125 * math.exp(-0.1 * t), 1.0 + math.exp(-(t - 3) ** 2), 0

    def a1(t):
        ke, en, _ = a0(t)
        return ke * (1 + 1e-6), en, 0

    _patch_gpu(monkeypatch, {"A-0": a0, "A-1": a1}, speed={"A-0": 40.0, "A-1": 41.0})
    rows = policy.long_run(["A-0", "A-1"], nel=2, N=3, re=2.0, dt=1e-3, t_end=6.0, projection=0,
                           chunk=50, every=10, cfl=0.4)
    r = {row["config"]: row for row in rows}
    a, b = r["A-0"], r["A-1"]
    assert 6.0 <= a["t_reached"] < 6.0 + 0.011 and a["stopped"] is None
    assert a["cfl_max"] == pytest.approx(0.4, rel=1e-12) and a["cfl_target"] == 0.4
    assert 0.009 < a["dt_mean"] < 0.01                 # 0.4 / 40, after the ramp from 1e-3
    assert a["energy_j"] == 250.0 and a["time_to_solution_s"] >= 0
    assert a["t_peak"] == pytest.approx(3.0, abs=2e-3)
    # A-1 steps at 0.4 / 41: its KE history, interpolated to A-0's times, is 1e-6
    # off (plus the linear interpolation's h^2/8 |KE''| / KE, about 1.3e-7)
    assert b["steps"] > a["steps"]
    assert abs(b["e_E_max"] - 1e-6) < 2e-7
    assert b["e_Omega_max"] < 1e-3


def test_peak_on_uneven_samples():
    """The vertex of the parabola through three unevenly spaced samples is exact
    for a parabola."""
    t = [0.0, 0.3, 0.5, 1.1, 1.2]
    tp, yp = policy.peak(t, [2 - 3 * (x - 0.61) ** 2 for x in t])
    assert tp == pytest.approx(0.61, abs=1e-12) and yp == pytest.approx(2.0, abs=1e-12)


def test_pressure_solver_option_reaches_the_stepper(monkeypatch):
    """replay() and long_run() with pressure="gmres_hsmg" switch every run's stepper to
    the GMRES + HSMG pressure solve (and leave it alone for "pcg"); the rows say which."""
    import math

    def a0(t):
        return 0.125 * math.exp(-t), 0.375 * (1 + t), 0

    _patch_gpu(monkeypatch, {"A-0": a0, "A-1": a0})
    from paper_2608_24348_gb300 import sem as sem_mod
    kinds = sem_mod.TGV.pressure_kinds
    policy.replay(["A-1"], nel=2, N=3, dt=0.01, steps=8, warm=3, pressure="gmres_hsmg")
    assert kinds == ["gmres_hsmg", "gmres_hsmg"]
    rows = policy.long_run(["A-0"], nel=2, N=3, re=2.0, dt=0.01, t_end=0.1, projection=0, chunk=5,
                           pressure="gmres_hsmg")
    assert kinds == ["gmres_hsmg"] * 3 and rows[0]["pressure"] == "gmres_hsmg"
    policy.long_run(["A-0"], nel=2, N=3, re=2.0, dt=0.01, t_end=0.1, projection=0, chunk=5)
    assert len(kinds) == 3
