"""Precision policies of the Taylor-Green stepper: the configurations of Table 2.

The paper's three-level model (Sec. 2, Fig. 2) maps (block, role, kernel, step
range) to a precision under a global cap rp.  The stepper exposes it through
``sem_tgv_set_policy``: per rule, the compute precision of the SEM block (the
dealiased convection), of the velocity block (three Helmholtz solves) and of
the pressure block (the Poisson solve), the storage cap, and the step the rule
starts at.  Accumulation (dots, norms, refinement residuals, BDF/EXT sums,
diagnostics) is FP64 in every configuration.

Readings of Table 2 on this stepper:
  - "fp32 compute" of a solve block: FP32 inner PCG inside FP64 iterative
    refinement to the block's own tolerance; "fp64 compute": PCG on the
    FP64-accurate operator;
  - the SEM block's compute precision applies to the dealiased convection (its
    hotspot, Fig. 3); the pointwise right-hand-side, divergence and gradient
    kernels stay FP64;
  - rp = fp32 (Group B): the stored state (velocity and convection histories,
    pressure) is rounded to FP32 values each step;
  - kernel-level fp16 overrides: adv_dealias = every operand of the convection's
    contractions rounded to FP16 with FP32 accumulation (B-5); ax_helm = the
    16-bit tensor-core operator in the inner PCG of the velocity (B-6) or the
    pressure (B-7) block.

Error metrics (Sec. 4.2, without the x100 %): e_E,max, e_Omega,max and
e_Omega,peak of a run's KE / enstrophy history against a reference history.
"""
from __future__ import annotations

import numpy as np

_A = dict(storage="f64")
_B = dict(storage="f32")

TABLE2 = {
    "A-0": dict(sem="f64", vel="f64", pres="f64", **_A),
    "A-1": dict(sem="f32", vel="f32", pres="f32", **_A),
    "A-2": dict(sem="f32", vel="f64", pres="f64", **_A),
    "A-3": dict(sem="f64", vel="f32", pres="f64", **_A),
    "A-4": dict(sem="f64", vel="f64", pres="f32", **_A),
    "B-0": dict(sem="f32", vel="f32", pres="f32", **_B),
    "B-1": dict(sem="f64", vel="f64", pres="f64", **_B),
    "B-2": dict(sem="f64", vel="f32", pres="f32", **_B),
    "B-3": dict(sem="f32", vel="f64", pres="f32", **_B),
    "B-4": dict(sem="f32", vel="f32", pres="f64", **_B),
    "B-5": dict(sem="f16_tc", vel="f32", pres="f32", **_B),
    "B-6": dict(sem="f32", vel="f16_tc", pres="f32", **_B),
    "B-7": dict(sem="f32", vel="f32", pres="f16_tc", **_B),
}


def rule(name: str, first_step: int = 1) -> dict:
    """The Table 2 configuration `name` as a policy rule starting at first_step."""
    return dict(TABLE2[name], first_step=first_step)


def e_max(hist, ref) -> float:
    """max_i |h_i - r_i| / max_i |r_i| (e_E,max and e_Omega,max of Sec. 4.2)."""
    h, r = np.asarray(hist, dtype=float), np.asarray(ref, dtype=float)
    return float(np.abs(h - r).max() / np.abs(r).max())


def e_peak(hist, ref) -> float:
    """|max_i h_i - max_i r_i| / max_i |r_i| (e_Omega,peak of Sec. 4.2)."""
    h, r = np.asarray(hist, dtype=float), np.asarray(ref, dtype=float)
    return float(abs(h.max() - r.max()) / np.abs(r).max())


def peak(t, y):
    """(time, value) of the largest sample of y(t), refined to the vertex of
    the parabola through it and its two neighbours (the samples may be
    unevenly spaced; the largest sample itself at either end of the record)."""
    t, y = np.asarray(t, dtype=float), np.asarray(y, dtype=float)
    k = int(np.argmax(y))
    if 0 < k < len(y) - 1:
        # parabola in s = t - t_k through (-h0, a), (0, b), (h1, c)
        h0, h1 = t[k] - t[k - 1], t[k + 1] - t[k]
        a, b, c = y[k - 1], y[k], y[k + 1]
        d0, d1 = (b - a) / h0, (c - b) / h1
        curv = (d1 - d0) / (h0 + h1)          # half the second derivative
        if curv < 0:
            slope = d0 + curv * h0            # first derivative at t_k
            off = -slope / (2 * curv)
            return float(t[k] + off), float(b + slope * off + curv * off * off)
    return float(t[k]), float(y[k])


def _errors(row, ref, uneven):
    """Sec. 4.2 metrics of row's KE / enstrophy history against ref's: step by
    step over the steps both reached, or (uneven: CFL-controlled steps, whose
    times differ between runs) with row's history interpolated linearly to
    ref's times within row's span."""
    if not uneven:
        n = min(len(row["ke"]), len(ref["ke"]))
        h_ke, h_en, r_ke, r_en = row["ke"][:n], row["enstrophy"][:n], ref["ke"][:n], ref["enstrophy"][:n]
    else:
        tr, t = np.asarray(ref["t"], dtype=float), np.asarray(row["t"], dtype=float)
        keep = (tr >= t[0]) & (tr <= t[-1])
        h_ke, h_en = np.interp(tr[keep], t, row["ke"]), np.interp(tr[keep], t, row["enstrophy"])
        r_ke, r_en = np.asarray(ref["ke"])[keep], np.asarray(ref["enstrophy"])[keep]
    return dict(e_E_max=e_max(h_ke, r_ke), e_Omega_max=e_max(h_en, r_en), e_Omega_peak=e_peak(h_en, r_en))


def replay(configs=None, nel=32, N=7, re=1600.0, dt=1e-3, steps=200, warm=3, maxit=4000, projection=0,
           cfl=None, pressure="pcg"):
    """Run each configuration from the same initial state on cuda:0; returns a
    list of dicts with ms/step of the timed steps (CUDA events around the
    graph replays and one copy of the stepper's log), the GPU energy of those
    steps from NVML's counter (energy_j, None where the counter is not
    readable), mean velocity / pressure
    iterations, the worst status and the error metrics of its KE / enstrophy
    history against A-0's.  pressure: "pcg" (Jacobi-PCG) or "gmres_hsmg" (the
    paper's GMRES + HSMG; direct launches).  cfl > 0 runs CFL-controlled steps from dt (one
    host synchronisation and direct launches per step; the rows then carry the
    mean step and CFL of the timed steps).  The first `warm`
    steps (startup orders and the graph capture) are part of the history but
    not of the timing; a configuration whose solves fail to converge within
    maxit iterations during them stops there (its row keeps the status).
    projection > 0 keeps that many earlier pressure solutions for the
    projection of each pressure solve (Sec. 3 uses 20)."""
    import math

    import torch

    from . import inputs, sem
    from .energy import EnergyMeter

    configs = list(configs or TABLE2)
    if "A-0" not in configs:
        configs = ["A-0"] + configs
    dev = torch.device("cuda:0")
    meter = EnergyMeter(0)
    ctx = sem.Ctx(N, (nel,) * 3, (2 * math.pi,) * 3, (1, 1, 1))
    xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.coords(xyz)
    x, y, z = xyz.view(3, -1)
    ic = [t.contiguous() for t in inputs.tgv_initial(x, y, z, lib=torch)]
    ic[2] = (ic[2] + 0 * x).contiguous()
    vo = sem.opts(tol=1e-6, abs_tol=True, maxit=maxit)
    po = sem.opts(tol=1e-4, abs_tol=True, maxit=maxit)
    out, ref = [], None
    for name in configs:
        T = sem.TGV(ctx, 1.0 / re, dt, op="f64", vel=vo, pres=po)
        T.set_policy([rule(name)])
        if projection:
            T.set_projection(projection)
        if pressure != "pcg":
            T.set_pressure_solver(pressure)
        T.set(*ic)
        if cfl:
            T.set_dt(cfl_target=cfl)
        stream = torch.cuda.Stream()
        joules = None
        with torch.cuda.stream(stream):
            d = T.step(warm, stream=stream)
            ms = float("nan")
            if all(r["status"] == 0 for r in d):  # a solve that fails to converge ends the run
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream.synchronize()
                meter.start()
                e0.record(stream)
                d += T.step(steps - warm, stream=stream)  # ends with one copy of the device log
                e1.record(stream)
                stream.synchronize()
                joules = meter.stop()
                ms = e0.elapsed_time(e1) / max(1, steps - warm)
        ke = [r["ke"] for r in d]
        en = [r["enstrophy"] for r in d]
        extra = {}
        if cfl:
            extra = dict(dt_mean=float(np.mean([r["dt"] for r in d[warm:]] or [np.nan])),
                         cfl_mean=float(np.mean([r["cfl"] for r in d[warm:]] or [np.nan])),
                         t_end=d[-1]["t"])
        row = dict(config=name, **TABLE2[name], projection=projection, ms_per_step=ms, energy_j=joules,
                   energy_reason=meter.reason, **extra,
                   vel_iters=float(np.mean([sum(r["iters"][1:]) / 3 for r in d])),
                   pres_iters=float(np.mean([r["iters"][0] for r in d])),
                   status=max((r["status"] for r in d), key=abs), ke=ke, enstrophy=en,
                   t=[r["t"] for r in d])
        if name == "A-0":
            ref = row
        out.append(row)
        T.close()
    meter.close()
    for row in out:
        row["steps"] = len(row["ke"])
        row.update(_errors(row, ref, bool(cfl)))
    return out


def long_run(configs=("A-0", "A-1", "B-0"), nel=32, N=7, re=1600.0, dt=4e-3, t_end=12.0, projection=20,
             chunk=250, warm=3, maxit=4000, every=25, budget_s=None, log=None, cfl=None, dt_max=None,
             pressure="pcg"):
    """Run each configuration from the Sec. 3 initial state to t_end (the long
    runs behind Table 3), in chunks of `chunk` graph-replayed steps; with
    cfl > 0 the steps are CFL-controlled from dt (Sec. 3 runs at CFL 0.4;
    capped by dt_max) and the run ends at the first step reaching t_end.
    pressure: "pcg" (Jacobi-PCG) or "gmres_hsmg" (GMRES + HSMG, Sec. 3).
    Time- and energy-to-solution cover every step (CUDA events; NVML's energy
    counter around the run, None where it is not readable).  A run stops
    early when a solve fails to converge, KE or enstrophy stop being finite or
    KE exceeds its initial value, or (budget_s) the configurations together
    have stepped for that many seconds.  Returns one dict per configuration:
    ms/step after the `warm` start-up steps, mean and largest iteration counts,
    the time reached, the enstrophy peak (time and value at the vertex of the
    parabola through the largest sample and its neighbours, and the dissipation rate
    2 nu Omega there), the dissipation rate -dKE/dt at the same time (their gap
    is the numerical dissipation of the discretisation), and the KE / enstrophy
    history every `every` steps; errors against A-0's history (Sec. 4.2) over
    the steps both reached.  log, if given, is called with a one-line summary
    after each configuration."""
    import math
    import time

    import torch

    from . import inputs, sem
    from .energy import EnergyMeter

    configs = list(configs)
    nu = 1.0 / re
    nsteps = int(round(t_end / dt))
    meter = EnergyMeter(0)
    ctx = sem.Ctx(N, (nel,) * 3, (2 * math.pi,) * 3, (1, 1, 1))
    xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=torch.device("cuda:0"))
    ctx.coords(xyz)
    x, y, z = xyz.view(3, -1)
    ic = [t.contiguous() for t in inputs.tgv_initial(x, y, z, lib=torch)]
    ic[2] = (ic[2] + 0 * x).contiguous()
    del xyz, x, y, z
    vo = sem.opts(tol=1e-6, abs_tol=True, maxit=maxit)
    po = sem.opts(tol=1e-4, abs_tol=True, maxit=maxit)
    wall0 = time.time()
    out = []
    for name in configs:
        T = sem.TGV(ctx, nu, dt, op="f64", vel=vo, pres=po)
        T.set_policy([rule(name)])
        if projection:
            T.set_projection(projection)
        if pressure != "pcg":
            T.set_pressure_solver(pressure)
        T.set(*ic)
        if cfl:
            T.set_dt(cfl_target=cfl, dt_max=dt_max or 0.0)
        ke0 = T.energy()[0]
        stream = torch.cuda.Stream()
        d, ms, timed, stop, ms_all = [], 0.0, 0, None, 0.0

        def more():
            if cfl:
                return not d or d[-1]["t"] < t_end * (1 - 1e-12)
            return len(d) < nsteps

        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            meter.start()
            while more():
                n = warm if not d else chunk
                if not cfl:
                    n = min(n, nsteps - len(d))
                e0.record(stream)
                part = T.step(n, stream=stream)
                e1.record(stream)
                stream.synchronize()
                if cfl:  # the run ends at the first step reaching t_end
                    k = next((i for i, r in enumerate(part) if r["t"] >= t_end * (1 - 1e-12)), None)
                    if k is not None:
                        part = part[:k + 1]
                ms_all += e0.elapsed_time(e1)
                if d:  # the start-up steps are not timed
                    ms += e0.elapsed_time(e1)
                    timed += n
                d += part
                if any(r["status"] != 0 for r in part):
                    stop = "solve status %d" % max((r["status"] for r in part), key=abs)
                elif not all(math.isfinite(r["ke"]) and math.isfinite(r["enstrophy"]) for r in part):
                    stop = "non-finite KE or enstrophy"
                elif max(r["ke"] for r in part) > ke0 * (1 + 1e-6):
                    stop = "KE above its initial value"
                elif budget_s is not None and time.time() - wall0 > budget_s:
                    stop = "time budget"
                if stop:
                    break
            stream.synchronize()
            joules = meter.stop()
        T.close()
        t = np.array([r["t"] for r in d])
        ke = np.array([r["ke"] for r in d])
        en = np.array([r["enstrophy"] for r in d])
        k = int(np.argmax(en))
        eps_ke = -np.gradient(ke, t) if len(t) > 2 else np.full_like(ke, np.nan)
        tp, ep = peak(t, en)
        out.append(dict(config=name, **TABLE2[name], re=re, dt=dt, nel=nel, N=N, projection=projection,
                        cfl_target=cfl, pressure=pressure, steps=len(d), t_reached=float(t[-1]) if len(t) else 0.0, stopped=stop,
                        ms_per_step=ms / timed if timed else float("nan"),
                        time_to_solution_s=ms_all / 1e3, energy_j=joules, energy_reason=meter.reason,
                        dt_mean=float(np.mean([r["dt"] for r in d])) if d else float("nan"),
                        cfl_max=float(max(r["cfl"] for r in d)) if d else float("nan"),
                        pres_iters=float(np.mean([r["iters"][0] for r in d])),
                        pres_iters_max=int(max(r["iters"][0] for r in d)),
                        vel_iters=float(np.mean([sum(r["iters"][1:]) / 3 for r in d])),
                        t_peak=tp, enstrophy_peak=ep,
                        eps_peak=float(2 * nu * en[k]), eps_ke_at_peak=float(eps_ke[k]),
                        ke_end=float(ke[-1]), ke=ke.tolist(), enstrophy=en.tolist(), t=t.tolist(),
                        series=[[float(t[i]), float(ke[i]), float(en[i])]
                                for i in range(every - 1, len(d), every)]))
        if log:
            r = out[-1]
            log("%s: %d steps to t=%.3f (%s), %.2f ms/step, pressure it. %.1f (max %d), "
                "enstrophy peak %.4f at t=%.3f" % (name, r["steps"], r["t_reached"], stop or "done",
                                                    r["ms_per_step"], r["pres_iters"], r["pres_iters_max"],
                                                    r["enstrophy_peak"], r["t_peak"]))
    meter.close()
    ref = next((r for r in out if r["config"] == "A-0"), None)
    for row in out:
        if ref is not None and row["steps"] and ref["steps"]:
            row.update(_errors(row, ref, bool(cfl)))
    for row in out:
        del row["ke"], row["enstrophy"], row["t"]
    return out


def main(argv=None):
    import argparse
    import json
    import sys

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nel", type=int, default=32)
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--re", type=float, default=1600.0)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--configs", default=",".join(TABLE2))
    ap.add_argument("--projection", type=int, default=0)
    ap.add_argument("--t-end", type=float, default=None,
                    help="run each configuration to this time instead (long runs; --projection "
                         "defaults to 20 there)")
    ap.add_argument("--budget-s", type=float, default=None)
    ap.add_argument("--cfl", type=float, default=None,
                    help="CFL-controlled steps from --dt towards this CFL number (Sec. 3: 0.4)")
    ap.add_argument("--dt-max", type=float, default=None)
    ap.add_argument("--pressure", default="pcg", choices=["pcg", "gmres_hsmg"])
    ap.add_argument("--out", default=None, help="long runs: write the rows with their histories here")
    args = ap.parse_args(argv)
    if args.t_end is not None:
        rows = long_run(args.configs.split(","), args.nel, args.N, args.re, args.dt, args.t_end,
                        projection=args.projection or 20, budget_s=args.budget_s,
                        log=lambda m: print(m, file=sys.stderr, flush=True), cfl=args.cfl,
                        dt_max=args.dt_max, pressure=args.pressure)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(rows, f)
        for r in rows:
            print(json.dumps({k: v for k, v in r.items() if k != "series"}), flush=True)
        return
    rows = replay(args.configs.split(","), args.nel, args.N, args.re, args.dt, args.steps,
                  projection=args.projection, cfl=args.cfl, pressure=args.pressure)
    for r in rows:
        r = {k: v for k, v in r.items() if k not in ("ke", "enstrophy", "t")}
        print(json.dumps(r))


if __name__ == "__main__":
    main()
