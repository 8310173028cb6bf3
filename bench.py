#!/usr/bin/env python3
"""Benchmark: sem_ax GDOF/s and PCG solve time at N=7 on 32^3 elements, FP64 vs mixed.

One step = one application of the Helmholtz operator sem_ax to the 16.8M-node
deformed mesh (32^3 elements, N=7, interior vertices perturbed by up to 10%,
u uniform in [-1,1] per unique node, h1 = 0.01, h2 = 1/dt with dt = 1e-3).
The primary value is the FP64 operator's throughput in GDOF/s (local nodes
per second) with the library's default FP64 path (FP64-accurate arithmetic on
the FP32 pipes).  Beside it: native-FP64, FP32 and BF16/FP16 tensor-core
operators, the FP64 and mixed-precision PCG solves of the pressure-Poisson
workload and an end-to-end (host buffers) figure.  Inputs (u 134 MB, geometry 940 MB) exceed the 129 MB L2,
so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ORDER, NEL, PERTURB, H1, H2 = 7, (32, 32, 32), 0.1, 0.01, 1000.0
METRIC = "sem_ax GDOF/s & PCG solve ms at N=7, 32^3 elems: mixed vs FP64, 1 GB300"
# algorithmic bytes per local node of one operator application
BYTES_F64 = 72  # read u 8 + G 48 + B 8, write w 8
BYTES_F32 = 36
# FP64 flops of one operator application per node: 12 (N+1) + 21 unfolded; the
# native kernel for even N+1 folds the contractions (even-odd split): 6 (N+1) + 21
FLOPS_PER_NODE = 6 * (N_ORDER + 1) + 21 if (N_ORDER + 1) % 2 == 0 else 12 * (N_ORDER + 1) + 21
# The FP64-accurate operator at N=7 is the block-floating-point kernel with u
# staged by bulk copies, one element per block (the library default):
# instructions per node from the ncu capture on the 24^3 mesh (all pipes),
# DRAM bytes per node from the same capture (453.33 MB read + 47.84 MB written
# for 7,077,888 nodes), scaled to the 32^3 mesh
DF_KERNEL = "k_ax_bfp_st<8,0,1,16>"
DF_INSTR_PER_NODE = 421
DF_TRAFFIC_PER_NODE = (453.33e6 + 47.84e6) / 7077888
FP64_PROBE_TFLOPS = 1.26  # FP64 FMA rate measured on this GPU model (probe: 2.2 FMA/clk/SM)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured",
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier_max(x, ws):
    """The largest x over the ws ranks (every rank gets it)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gdofs(nodes_per_rank, seconds_max, ws):
    """Whole-job throughput: every rank's replica, over the slowest rank's time."""
    return ws * nodes_per_rank / seconds_max / 1e9


def cpu_baseline(seconds=12.0, threads=None, edge=16):
    """The FP64 oracle's operator on the host cores, on an edge^3-element sample
    of the same deformed N=7 mesh, repeated for about `seconds` (threads: the
    OpenMP thread count, default all cores)."""
    import numpy as np

    import oracle
    from paper_2608_24348_gb300 import inputs
    full = os.cpu_count() or 1
    oracle.set_threads(threads or full)
    nel = (edge, edge, edge)
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=PERTURB)
    m = oracle.Mesh(N_ORDER, nel, v)
    u = inputs.unique_uniform_field(N_ORDER, nel, seed=inputs.SEED_FIELD)
    m.ax(u, H1, H2)
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < seconds or reps < 1:
        m.ax(u, H1, H2)
        reps += 1
    dt = time.perf_counter() - t0
    used = oracle.threads()
    oracle.set_threads(full)
    return {"value": m.nL * reps / dt / 1e9, "unit": "GDOF/s", "cores": used,
            "kind": "oracle",
            "sample": f"FP64 oracle sem_ax on a {edge}^3-element N=7 deformed mesh "
                      f"({m.nL} nodes), {reps} applications in {dt:.1f} s"}, reps, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per = max(2.0, min(20.0, 60.0 / max(1, args.steps)))
    vals = []
    info = None
    for _ in range(args.warmup):
        cpu_baseline(seconds=0.5)
    t_all = time.perf_counter()
    for _ in range(args.steps):
        info, reps, dt = cpu_baseline(seconds=per)
        vals.append(info["value"])
    wall = time.perf_counter() - t_all
    v = statistics.median(vals)
    cb = dict(info)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sem_ax, 16^3-element sample of the 32^3 N=7 deformed mesh "
                                   "(FP64 CPU oracle)", "N": N_ORDER},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_kernel(fn, steps, warmup, stream, ws):
    """Events around every step on `stream`; barrier + sync on both sides."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            fn()
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total = ev[0].elapsed_time(ev[steps])
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    return per, total


def pcg_section(ctx, sem, inputs, stream, ws, reps=1):
    """Pressure Poisson on the same mesh: RHS = div of a seeded random smooth
    field (|k| <= 8); FP64 Jacobi-PCG vs FP32-inner / FP64 refinement, both to
    the FP64 relative residual 1e-10.  Each solve is one persistent launch,
    timed with CUDA events on the launching stream (best of `reps`)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.coords(xyz)
    K, cc, cs = inputs.fourier_div_modes()
    f = inputs.eval_fourier(K, cc, cs, *xyz.view(3, -1))
    b = torch.empty_like(f)
    ctx.ax(f, b, 0.0, 1.0, "f64")
    ctx.dssum(b, "f64")
    del xyz, f
    out = {"workload": "pressure Poisson, 32^3 N=7 deformed, RHS div of random smooth field "
                       "|k|<=8, h1=1 h2=0, rel tol 1e-10; relres_native = true residual of the "
                       "solution under the native FP64 operator"}
    sp = stream.cuda_stream
    ones = torch.ones_like(b)
    ctx.dssum(ones, "f64")
    imult = 1.0 / ones
    del ones

    def relres_native(x):
        w = torch.empty_like(x)
        ctx.ax(x, w, 1.0, 0.0, "f64_native", stream=sp)
        ctx.dssum(w, "f64", stream=sp)
        bm = b - (b * imult).sum() / imult.sum()
        r = bm - w
        return float(torch.sqrt((r * r * imult).sum() / (bm * bm * imult).sum()))

    for name, kw in (("fp64", {}), ("fp64_native", {"inner": "f64_native"}),
                     ("mixed_f32", {"inner": "f32", "inner_tol": 1e-4}),
                     ("mixed_bf16_tc", {"inner": "bf16_tc", "inner_tol": 1e-2}),
                     ("mixed_f16x2_tc", {"inner": "f16x2_tc", "inner_tol": 1e-4}),
                     ("mixed_bf16x3_tc", {"inner": "bf16x3_tc", "inner_tol": 1e-4})):
        best = None
        info = None
        for _ in range(reps):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.pcg_solve(b, x, 1.0, 0.0, sync=False, stream=sp, tol=1e-10, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            info = ctx.last_solve_info()
            best = ms if best is None else min(best, ms)
        out[name] = {"ms": barrier_max(best, ws), "iters": info["iters"],
                     "outer": info["outer_iters"], "status": info["status"],
                     "relres": info["rnorm"] / info["bnorm"] if info["bnorm"] else None}
        if name in ("fp64", "mixed_f32"):
            out[name]["relres_native"] = relres_native(x)
    # the paper's pressure solver: flexible GMRES(30) with the hybrid Schwarz
    # multigrid (orders 7, 3, 1; coarse Jacobi-PCG to 1e-1), V-cycle in FP32 or
    # FP64; one-off setup timed apart; the solve syncs the host every iteration
    import time
    for name, vdt in (("gmres_hsmg_f32", "f32"), ("gmres_hsmg_f64", "f64")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = sem.HSMG(ctx, [7, 3, 1], dtype=vdt, coarse_tol=0.1)
        setup_ms = (time.perf_counter() - t0) * 1e3
        best, info = None, None
        for _ in range(max(reps, 2)):   # the first solve also allocates the Krylov basis
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = H.gmres(b, x, restart=30, stream=sp, tol=1e-10)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        H.close()
        out[name] = {"ms": barrier_max(best, ws), "iters": info["iters"], "restarts": info["outer_iters"],
                     "status": info["status"], "setup_ms": setup_ms,
                     "relres": info["rnorm"] / info["bnorm"] if info["bnorm"] else None,
                     "relres_native": relres_native(x)}
    out["speedup_mixed_f32_vs_fp64"] = out["fp64"]["ms"] / out["mixed_f32"]["ms"]
    out["speedup_mixed_f32_vs_fp64_native"] = out["fp64_native"]["ms"] / out["mixed_f32"]["ms"]
    out["speedup_gmres_hsmg_f32_vs_fp64_pcg"] = out["fp64"]["ms"] / out["gmres_hsmg_f32"]["ms"]
    return out


def plain_poisson_section(sem, inputs, stream, reps=20):
    """The plain FP64 Poisson workload: periodic [0, 2 pi]^3, 4x4x4 undeformed
    elements, N=5, f = 3 sin x sin y sin z (b = dssum(B f), its mean removed by
    the solver), Jacobi-PCG with the FP64-accurate operator to the relative
    residual 1e-10 from x0 = 0.  Median of `reps` solves (CUDA events on the
    launching stream) and the nodal max error against u* = sin x sin y sin z."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = sem.Ctx(5, (4, 4, 4), (2 * math.pi,) * 3, (1, 1, 1))
    xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.coords(xyz)
    x, y, z = xyz.view(3, -1)
    us = torch.sin(x) * torch.sin(y) * torch.sin(z)
    b = torch.empty_like(us)
    ctx.ax(3.0 * us, b, 0.0, 1.0, "f64", stream=stream.cuda_stream)
    ctx.dssum(b, "f64", stream=stream.cuda_stream)
    sol = torch.zeros_like(b)
    times = []
    for _ in range(reps):
        sol.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.pcg_solve(b, sol, 1.0, 0.0, sync=False, stream=stream.cuda_stream, tol=1e-10)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    info = ctx.last_solve_info()
    err = float((sol - us).abs().max())
    ctx.close()
    return {"workload": "plain FP64 Poisson: periodic [0,2pi]^3, 4x4x4 undeformed, N=5, "
                        "f=3 sin x sin y sin z, rel tol 1e-10", "ms_median": statistics.median(times),
            "iters": info["iters"], "status": info["status"],
            "relres": info["rnorm"] / info["bnorm"] if info["bnorm"] else None,
            "max_err_vs_exact": err}


def batched_section(sem, inputs, stream, peak_gbs):
    """The uneven batch: 64 periodic Poisson problems (E in {8^3 .. 24^3}, N in
    {5, 7, 9}, sine RHS with seeded wavenumbers) solved in one persistent launch,
    an FP32-accurate inner PCG inside FP64 refinement to 1e-10, each order's
    inner path (FP32 CUDA cores or split FP16 tensor cores) chosen by the tuner.  Throughput counts each
    problem's inner iterations times its local nodes; the HBM fraction counts
    84 bytes per local node and inner iteration (the FP32 iteration's streams)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    specs = inputs.batch_problems()
    ctxs, bs, xs = [], [], []
    for (edge, N, k1, k2, k3) in specs:
        ctx = sem.Ctx(N, (edge,) * 3, (2 * math.pi,) * 3, (1, 1, 1))
        xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
        ctx.coords(xyz)
        kk = float(k1 * k1 + k2 * k2 + k3 * k3)
        f = kk * inputs.sine_product((k1, k2, k3), *xyz.view(3, -1), lib=torch)
        b = torch.empty_like(f)
        ctx.ax(f, b, 0.0, 1.0, "f64")
        ctx.dssum(b, "f64")
        del xyz, f
        ctxs.append(ctx)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    n = len(ctxs)
    # per-order inner path (FP32 CUDA cores or split FP16 tensor cores) chosen by
    # the tuner on one context of each order
    tuned = {}
    for (edge, N, *_), c in zip(specs, ctxs):
        if N not in tuned:
            tuned[N] = sem.tune_inner(c, iters=20)
    kw = dict(tol=1e-10, inner="f32_tuned", inner_tol=1e-4)
    sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * n, [0.0] * n, **kw)  # warm-up (Jacobi inverses)
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # synchronous call: returns once the launch has finished and the infos are filled
    infos = sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * n, [0.0] * n, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nodes = sum(c.nL for c in ctxs)
    work = sum(i["iters"] * c.nL for i, c in zip(infos, ctxs))
    gbs = 84.0 * work / (ms * 1e-3) / 1e9
    out = {"workload": "64 uneven periodic Poisson problems, E in {8^3..24^3}, N in {5,7,9}, "
                       "FP32-accurate inner (per-order path chosen by the tuner) / FP64 refinement "
                       "to 1e-10, one persistent launch",
           "ms": ms, "local_nodes": nodes, "inner_iters_total": sum(i["iters"] for i in infos),
           "status_all_ok": all(i["status"] == 0 for i in infos),
           "gdofs_iter": work / (ms * 1e-3) / 1e9, "hbm_gbs": gbs, "hbm_frac": gbs / peak_gbs,
           "tile": {str(N): {"inner_path": "fp16x2_tensor_cores" if t["path"] else "fp32_cuda_cores",
                             "elements_per_block": 8 if t["path"] else 256 // (N + 1) ** 2,
                             "ms_per_inner_iter": t["ms_per_iter"]}
                    for N, t in sorted(tuned.items())},
           "threads_per_block": 256}
    for c in ctxs:
        c.close()
    return out


def tgv_replay_section(steps=200):
    """Taylor-Green vortex Re=1600, 32^3 undeformed, N=7, dt=1e-3: 200 steps of the
    FP64 (A-0) and FP32-compute (A-1) policies of Table 2 from the Sec. 3 initial
    state, the pressure solve projected onto 20 previous solutions; ms per
    graph-replayed step (CUDA events around the steps after the first three)
    and the Sec. 4.2 errors of A-1's KE / enstrophy history against A-0's."""
    from paper_2608_24348_gb300 import policy
    rows = policy.replay(configs=["A-0", "A-1"], steps=steps, projection=20)
    ref = rows[0]
    out = {"workload": f"TGV Re=1600, 32^3 undeformed, N=7, dt=1e-3, {steps} steps, projection 20, "
                       "BDF3/EXT3 with 3/2 dealiasing; ms per graph-replayed step after 3; GPU "
                       "energy of those steps from NVML's counter"}
    for r in rows:
        out[r["config"]] = {"ms_per_step": r["ms_per_step"], "pres_iters": r["pres_iters"],
                            "vel_iters": r["vel_iters"], "status": r["status"],
                            "ke_last": r["ke"][-1], "enstrophy_last": r["enstrophy"][-1],
                            "e_E_max": r["e_E_max"], "e_Omega_max": r["e_Omega_max"],
                            "e_Omega_peak": r["e_Omega_peak"], "energy_j": r["energy_j"],
                            "j_per_step": (r["energy_j"] / (r["steps"] - 3)
                                           if r["energy_j"] is not None else None)}
        if r["energy_j"] is None:
            out[r["config"]]["energy_unavailable"] = r["energy_reason"]
    # the paper's pressure solver (GMRES + HSMG) in the same A-0 run: direct
    # launches (GMRES reads back to the host), errors against the Jacobi-PCG run
    g = policy.replay(configs=["A-0"], steps=steps, projection=20, pressure="gmres_hsmg")[0]
    out["A-0_gmres_hsmg"] = {"ms_per_step": g["ms_per_step"], "pres_iters": g["pres_iters"],
                             "vel_iters": g["vel_iters"], "status": g["status"], "energy_j": g["energy_j"],
                             "e_E_max_vs_pcg": policy.e_max(g["ke"], ref["ke"]),
                             "e_Omega_max_vs_pcg": policy.e_max(g["enstrophy"], ref["enstrophy"])}
    # CFL-controlled steps (Sec. 3: CFL 0.4) from the same state: one host
    # synchronisation and direct launches per step
    n_cfl = max(20, steps // 2)
    rows = policy.replay(configs=["A-0", "A-1"], steps=n_cfl, projection=20, cfl=0.4)
    out["cfl_0.4"] = {"workload": f"the same start, {n_cfl} CFL-controlled steps from dt=1e-3 "
                                  "(variable-step BDF3/EXT3), ms per step after 3"}
    for r in rows:
        out["cfl_0.4"][r["config"]] = {
            "ms_per_step": r["ms_per_step"], "dt_mean": r.get("dt_mean"), "cfl_mean": r.get("cfl_mean"),
            "t_end": r.get("t_end"), "pres_iters": r["pres_iters"], "status": r["status"],
            "e_E_max": r["e_E_max"], "e_Omega_max": r["e_Omega_max"], "energy_j": r["energy_j"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2608_24348_gb300 import inputs, sem

    dev = torch.device("cuda", local)
    pk = peaks()
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    v = inputs.box_vertices(NEL, (2 * math.pi,) * 3, perturb=PERTURB)
    ctx = sem.Ctx(N_ORDER, NEL, (2 * math.pi,) * 3, (1, 1, 1), vertices=v)
    nL = ctx.nL
    u_h = inputs.unique_uniform_field(N_ORDER, NEL, seed=inputs.SEED_FIELD)
    u64 = torch.from_numpy(u_h).to(dev)
    w64 = torch.empty_like(u64)
    u32 = u64.float()
    w32 = torch.empty_like(u32)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream

    def run(dt, x, y):
        return lambda: ctx.ax(x, y, H1, H2, dt, stream=sp)

    clocks = Clocks(local)
    clocks.start()
    per64, tot64 = time_kernel(run("f64", u64, w64), args.steps, args.warmup, stream, ws)
    k2 = max(20, args.steps // 5)
    per_nat, tot_nat = time_kernel(run("f64_native", u64, w64), k2, 3, stream, ws)
    per32, tot32 = time_kernel(run("f32", u32, w32), args.steps, args.warmup, stream, ws)
    per_bf, tot_bf = time_kernel(run("bf16_tc", u32, w32), k2, 3, stream, ws)
    per_f16, tot_f16 = time_kernel(run("f16_tc", u32, w32), k2, 3, stream, ws)
    _, tot_f16x2 = time_kernel(run("f16x2_tc", u32, w32), k2, 3, stream, ws)
    _, tot_bf16x3 = time_kernel(run("bf16x3_tc", u32, w32), k2, 3, stream, ws)
    pcg = pcg_section(ctx, sem, inputs, stream, ws)
    plain = plain_poisson_section(sem, inputs, stream)
    clk = clocks.stop()

    tot64 = barrier_max(tot64, ws)
    ms64 = tot64 / args.steps
    gdof = lambda ms: aggregate_gdofs(nL, ms * 1e-3, ws)
    avg64 = statistics.mean(per64)
    mhz = clk.get("sm_max_mhz") or pk["sm_max_mhz"]
    fp32_peak = 128 * n_sms * mhz * 1e6 / 1e12          # FP32-pipe ops/s (T)
    fp64_peak = FP64_PROBE_TFLOPS
    df_ops = DF_INSTR_PER_NODE * nL / (avg64 * 1e-3) / 1e12
    avg_nat = statistics.mean(per_nat)
    avg32 = statistics.mean(per32)
    hbm = lambda B, ms: B * nL / (ms * 1e-3) / 1e9

    # end to end through the C ABI with pinned host buffers: u comes from and w
    # returns to host memory inside every call (the FP64-accurate operator reads
    # and writes the mapped host memory over the host link itself)
    uh = torch.from_numpy(u_h).pin_memory()
    wh = torch.empty_like(uh).pin_memory()
    ctx.ax(uh, wh, H1, H2, "f64", stream=sp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = 20
    for _ in range(ne):
        ctx.ax(uh, wh, H1, H2, "f64", stream=sp)
    torch.cuda.synchronize()
    e2e_s = barrier_max((time.perf_counter() - t0) / ne, ws)

    line = {
        "metric": METRIC, "value": gdof(ms64), "unit": "GDOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "df64", "data": "synthetic",
        "config": {"workload": "sem_ax FP64 (FP64-accurate, FP32 pipes), 32^3 elements N=7 "
                               "deformed (16.8M local nodes), h1=0.01 h2=1000", "N": N_ORDER,
                   "elements": list(NEL), "local_nodes": nL,
                   "l2": "inputs larger than L2 (1.2 GB per application), no flush"},
        "roofline": {"bound": "hbm", "achieved": hbm(BYTES_F64, avg64), "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": hbm(BYTES_F64, avg64) / pk["hbm_gbs"],
                     "traffic": DF_TRAFFIC_PER_NODE * nL, "peak_src": pk["src"],
                     "kernel": DF_KERNEL, "bytes_per_node": BYTES_F64,
                     "issue": {"achieved": df_ops, "peak": fp32_peak, "unit": "T thread-instr/s",
                               "frac": df_ops / fp32_peak, "instr_per_node": DF_INSTR_PER_NODE,
                               "peak_src": "one warp instruction per clock per SM sub-partition "
                                           "(128 thread-instr/clk/SM) x SMs x max SM clock"}},
        "native_f64": {"gdofs": gdof(barrier_max(tot_nat, ws) / k2),
                       "roofline": {"bound": "alu", "unit": "TFLOP/s", "kernel": "k_ax_eo64<8>",
                                    "flops_per_node": FLOPS_PER_NODE,
                                    "achieved": FLOPS_PER_NODE * nL / (avg_nat * 1e-3) / 1e12,
                                    "peak": fp64_peak, "peak_src": "FP64 FMA probe",
                                    "frac": FLOPS_PER_NODE * nL / (avg_nat * 1e-3) / 1e12 / fp64_peak,
                                    "hbm_frac": hbm(BYTES_F64, avg_nat) / pk["hbm_gbs"]}},
        "mixed": {"sem_ax_f32_gdofs": gdof(barrier_max(tot32, ws) / args.steps),
                  "roofline": {"bound": "hbm", "achieved": hbm(BYTES_F32, avg32),
                               "peak": pk["hbm_gbs"], "unit": "GB/s",
                               "frac": hbm(BYTES_F32, avg32) / pk["hbm_gbs"]},
                  "sem_ax_bf16_tc_gdofs": gdof(barrier_max(tot_bf, ws) / k2),
                  "sem_ax_f16_tc_gdofs": gdof(barrier_max(tot_f16, ws) / k2),
                  "sem_ax_f16x2_tc_gdofs": gdof(barrier_max(tot_f16x2, ws) / k2),
                  "sem_ax_bf16x3_tc_gdofs": gdof(barrier_max(tot_bf16x3, ws) / k2)},
        "pcg": pcg,
        "plain_poisson": plain,
        "e2e": {"value": ws * nL / e2e_s / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": 8 * nL,
                "d2h_bytes_per_step": 8 * nL},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    # the batch and the Taylor-Green replay run after the timed operator (their
    # own CUDA events); the 32^3 context is released first
    del u64, w64, u32, w32
    ctx.close()
    torch.cuda.empty_cache()
    line["batched"] = batched_section(sem, inputs, stream, pk["hbm_gbs"])
    torch.cuda.empty_cache()
    line["tgv"] = tgv_replay_section()
    if rank == 0:
        cb, _, _ = cpu_baseline(seconds=12.0)
        cb1, _, _ = cpu_baseline(seconds=4.0, threads=1, edge=8)
        cb["value_1thread"] = cb1["value"]
        cb["sample_1thread"] = cb1["sample"]
        line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
