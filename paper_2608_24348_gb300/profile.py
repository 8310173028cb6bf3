"""Run one hot kernel on a chosen mesh, for profiler captures (ncu) of a small case.

    python -m paper_2608_24348_gb300.profile --kernel ax_f64 --nel 24 --reps 3

Kernels: ax_f64, ax_f64_native, ax_f32, ax_bf16_tc, dssum, pcg_f64, pcg_f32 (a
bounded number of PCG iterations), gmres_hsmg (a bounded number of GMRES
iterations with the hybrid Schwarz multigrid, FP32 V-cycle), tgv_f64, tgv_f32
(steps of the Taylor-Green stepper; --gmres for the GMRES + HSMG pressure
solve).
The mesh is the benchmark's: nel^3 elements, order N, interior vertices
perturbed by up to 10%.  --variant selects sem_ax's kernel candidate for the
order and dtype (see sem_tune_ax; default: the built-in choice).
"""
from __future__ import annotations

import argparse
import math


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default="ax_f64")
    ap.add_argument("--nel", type=int, default=24)
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--maxit", type=int, default=20)
    ap.add_argument("--projection", type=int, default=0, help="TGV: pressure projection space")
    ap.add_argument("--variant", type=int, default=-1, help="sem_ax kernel candidate (-1: default)")
    ap.add_argument("--gmres", action="store_true", help="TGV: GMRES + HSMG pressure solver")
    args = ap.parse_args(argv)

    import json
    import time

    import torch

    from . import inputs, sem
    dev = torch.device("cuda:0")
    nel = (args.nel,) * 3
    tgv = args.kernel.startswith("tgv")
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=0.0 if tgv else 0.1)
    ctx = sem.Ctx(args.N, nel, (2 * math.pi,) * 3, (1, 1, 1), vertices=v)
    u = torch.from_numpy(inputs.unique_uniform_field(args.N, nel)).to(dev)
    if args.kernel.startswith("ax") or args.kernel == "dssum":
        dt = args.kernel[3:] if args.kernel.startswith("ax") else "f64"
        if args.variant >= 0:
            sem.set_ax_variant(args.N, dt, args.variant)
        x = u if dt.startswith("f64") else u.float()
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
    elif args.kernel == "gmres_hsmg":
        b = torch.empty_like(u)
        ctx.ax(u, b, 0.0, 1.0, "f64")
        ctx.dssum(b, "f64")
        H = sem.HSMG(ctx, [args.N, 3, 1], dtype="f32", coarse_tol=0.1)
        for _ in range(args.reps):
            x = torch.zeros_like(b)
            H.gmres(b, x, restart=30, tol=1e-14, maxit=args.maxit)
    elif tgv:
        x, y, z = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev).view(3, -1)
        xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
        ctx.coords(xyz)
        x, y, z = xyz.view(3, -1)
        uu, vv, ww, pp = inputs.tgv_initial(x, y, z, lib=torch)
        T = sem.TGV(ctx, 1.0 / 1600, 1e-3, op=args.kernel[4:])
        if args.projection:
            T.set_projection(args.projection)
        if args.gmres:
            T.set_pressure_solver("gmres_hsmg")
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
