"""Run one hot kernel on a chosen mesh, for profiler captures (ncu) of a small case.

    python -m paper_2608_24348_gb300.profile --kernel ax_f64 --nel 24 --reps 3

Kernels: ax_f64, ax_f32, ax_bf16_tc, dssum, pcg_f64, pcg_f32 (a bounded number
of PCG iterations), tgv_f64, tgv_f32 (steps of the Taylor-Green stepper).
The mesh is the benchmark's: nel^3 elements, order N, interior vertices
perturbed by up to 10%.

--kernel link times the host link instead (no library call): copies of one
FP64 E-vector of the nel^3, order-N mesh between pinned host memory and the
device, host-to-device alone, device-to-host alone and both at once on two
streams, in GB/s per direction (the ceiling of the end-to-end sem_ax figure).
"""
from __future__ import annotations

import argparse
import math


def link_bandwidth(n, reps):
    """GB/s per direction of n-double copies between pinned host memory and
    cuda:0: host-to-device, device-to-host, and both concurrently."""
    import torch
    dev = torch.device("cuda:0")
    a_h = torch.ones(n, dtype=torch.float64).pin_memory()
    b_h = torch.empty(n, dtype=torch.float64).pin_memory()
    a_d = torch.empty(n, dtype=torch.float64, device=dev)
    b_d = torch.ones(n, dtype=torch.float64, device=dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def h2d():
        a_d.copy_(a_h, non_blocking=True)

    def d2h():
        b_h.copy_(b_d, non_blocking=True)

    def both():
        cur = torch.cuda.current_stream()
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            a_d.copy_(a_h, non_blocking=True)
        with torch.cuda.stream(s2):
            b_h.copy_(b_d, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    out = {"bytes_per_direction": 8 * n}
    for name, fn in (("h2d", h2d), ("d2h", d2h), ("both", both)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "GBps_per_direction": 8 * n / ms / 1e6}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default="ax_f64")
    ap.add_argument("--nel", type=int, default=24)
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--maxit", type=int, default=20)
    ap.add_argument("--projection", type=int, default=0, help="TGV: pressure projection space")
    args = ap.parse_args(argv)

    import json
    import time

    import torch

    from . import inputs, sem
    dev = torch.device("cuda:0")
    if args.kernel == "link":
        print(json.dumps(link_bandwidth(args.nel ** 3 * (args.N + 1) ** 3, max(args.reps, 3))))
        return
    nel = (args.nel,) * 3
    tgv = args.kernel.startswith("tgv")
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=0.0 if tgv else 0.1)
    ctx = sem.Ctx(args.N, nel, (2 * math.pi,) * 3, (1, 1, 1), vertices=v)
    u = torch.from_numpy(inputs.unique_uniform_field(args.N, nel)).to(dev)
    if args.kernel.startswith("ax") or args.kernel == "dssum":
        dt = args.kernel[3:] if args.kernel.startswith("ax") else "f64"
        x = u if dt == "f64" else u.float()
        w = torch.empty_like(x)
        for _ in range(args.reps):
            if args.kernel == "dssum":
                ctx.dssum(x, "f64")
            else:
                ctx.ax(x, w, 0.01, 1000.0, dt)
    elif args.kernel.startswith("pcg"):
        b = torch.empty_like(u)
        ctx.ax(u, b, 0.0, 1.0, "f64")
        ctx.dssum(b, "f64")
        for _ in range(args.reps):
            x = torch.zeros_like(b)
            ctx.pcg_solve(b, x, 1.0, 0.0, tol=1e-14, maxit=args.maxit,
                          inner=args.kernel[4:], inner_tol=1e-4)
    elif tgv:
        x, y, z = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev).view(3, -1)
        xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
        ctx.coords(xyz)
        x, y, z = xyz.view(3, -1)
        uu, vv, ww, pp = inputs.tgv_initial(x, y, z, lib=torch)
        T = sem.TGV(ctx, 1.0 / 1600, 1e-3, op=args.kernel[4:])
        if args.projection:
            T.set_projection(args.projection)
        T.set(uu.contiguous(), vv.contiguous(), (ww + 0 * x).contiguous(), pp.contiguous())
        T.step(3)  # startup orders 1, 2 and the first third-order step (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = T.step(args.reps)
        dt = time.perf_counter() - t0
        print(json.dumps({"tgv": args.kernel, "nL": ctx.nL, "steps": args.reps,
                          "ms_per_step": 1e3 * dt / args.reps,
                          "iters_last": d[-1]["iters"], "ke_last": d[-1]["ke"],
                          "enstrophy_last": d[-1]["enstrophy"],
                          "status": [r["status"] for r in d][-1]}))
    else:
        raise SystemExit(f"unknown kernel {args.kernel}")
    torch.cuda.synchronize()
    print("done", args.kernel, ctx.nL)


if __name__ == "__main__":
    main()
