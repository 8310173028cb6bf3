"""Batched uneven solves: many independent periodic Poisson problems in one
persistent launch (FP32 inner PCG, FP64 refinement to 1e-10), and the same
batch captured in a CUDA graph.

Bars: every problem's FP64 relative residual, evaluated by the oracle's
operator, <= 1.5e-10; on seeded problems the solution matches the oracle
solved to 1e-12 within 1e-9.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import pair, rel, sine_rhs, torch_dev
from paper_2608_24348_gb300 import inputs

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def _problems(sem, specs):
    ctxs, bs, xs, meta = [], [], [], []
    torch, dev = torch_dev()
    for (edge, N, k1, k2, k3) in specs:
        ctx, _, _ = pair(sem, N, (edge,) * 3, 0.0, with_oracle=False)
        bg, _, _ = sine_rhs(ctx, None, (k1, k2, k3))
        ctxs.append(ctx)
        bs.append(bg)
        xs.append(torch.zeros_like(bg))
        meta.append((edge, N, (k1, k2, k3)))
    return ctxs, bs, xs, meta


def _oracle_check(meta_i, x, full_solve=False):
    edge, N, k = meta_i
    v = inputs.box_vertices((edge,) * 3, (TWO_PI,) * 3)
    m = oracle.Mesh(N, (edge,) * 3, v)
    us = inputs.sine_product(k, *m.xyz)
    bo = m.dssum(m.B * float(sum(c * c for c in k)) * us)
    r, bn = m.residual(bo, x, 1.0, 0.0)
    assert r <= 1.5e-10 * bn, (meta_i, r, bn)
    if full_solve:
        xt, _ = m.pcg(bo, 1.0, 0.0, tol=1e-12)
        assert rel(x, xt) <= 1e-9, meta_i


def test_small_uneven_batch_matches_oracle(sem):
    specs = [(3, 5, 1, 2, 1), (2, 7, 1, 1, 1), (2, 9, 2, 1, 1), (4, 5, 1, 1, 2), (3, 7, 2, 2, 1)]
    ctxs, bs, xs, meta = _problems(sem, specs)
    infos = sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * len(ctxs), [0.0] * len(ctxs), tol=1e-10,
                                  inner="f32", inner_tol=1e-4)
    for i, info in enumerate(infos):
        assert info["status"] == 0, (meta[i], info)
        _oracle_check(meta[i], xs[i].cpu().numpy(), full_solve=True)
    # the same problems solved one by one give the same solutions
    for i, ctx in enumerate(ctxs):
        torch, _ = torch_dev()
        x1 = torch.zeros_like(bs[i])
        assert ctx.pcg_solve(bs[i], x1, tol=1e-10, inner="f32", inner_tol=1e-4)["status"] == 0
        assert rel(x1.cpu().numpy(), xs[i].cpu().numpy()) <= 1e-9


def test_repeated_context_in_a_batch(sem):
    """One context used by three problems (as the stepper's velocity solves)."""
    torch, dev = torch_dev()
    ctx, m, _ = pair(sem, 5, (3, 3, 2), 0.1)
    rhs = [sine_rhs(ctx, m, k) for k in ((1, 1, 1), (2, 1, 1), (1, 1, 3))]
    xs = [torch.zeros_like(r[0]) for r in rhs]
    infos = sem.pcg_solve_batched([ctx] * 3, [r[0] for r in rhs], xs, [1.0] * 3, [2.0] * 3,
                                  tol=1e-10)
    for i in range(3):
        assert infos[i]["status"] == 0
        r, bn = m.residual(rhs[i][1], xs[i].cpu().numpy(), 1.0, 2.0)
        assert r <= 1.5e-10 * bn


def test_batched_solve_in_a_cuda_graph(sem):
    torch, dev = torch_dev()
    specs = [(3, 5, 1, 2, 1), (2, 7, 1, 1, 1), (2, 9, 2, 1, 1)]
    ctxs, bs, xs, meta = _problems(sem, specs)
    ref = [torch.zeros_like(b) for b in bs]
    sem.pcg_solve_batched(ctxs, bs, ref, [1.0] * 3, [0.0] * 3, tol=1e-10, inner="f32")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up on the capture stream
        sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * 3, [0.0] * 3, sync=False, tol=1e-10, inner="f32")
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for x in xs:
            x.zero_()
        sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * 3, [0.0] * 3, sync=False, tol=1e-10,
                              inner="f32")
    for _ in range(2):
        for x in xs:
            x.fill_(7.0)
        g.replay()
        torch.cuda.synchronize()
        for i in range(3):
            assert rel(xs[i].cpu().numpy(), ref[i].cpu().numpy()) <= 1e-12


def test_uneven_batch_of_64_in_one_launch(sem):
    """The 64-problem uneven batch: E in {8^3 .. 24^3}, N in {5, 7, 9}, sine RHS
    with wavenumbers 1..4; every residual checked by the oracle's operator,
    four seeded problems solved by the oracle as well."""
    torch, dev = torch_dev()
    specs = inputs.batch_problems()
    ctxs, bs, xs, meta = _problems(sem, specs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * 64, [0.0] * 64, tol=1e-10, inner="f32",
                                  inner_tol=1e-4)
    e1.record()
    torch.cuda.synchronize()
    nodes = sum(c.nL for c in ctxs)
    iters = [i["iters"] for i in infos]
    print(f"\nbatch of 64: {nodes} local nodes, {e0.elapsed_time(e1):.1f} ms, "
          f"inner iterations {min(iters)}..{max(iters)}")
    assert all(i["status"] == 0 for i in infos), [i["status"] for i in infos]
    rng = np.random.default_rng(inputs.SEED_BATCH)
    small = [i for i, m in enumerate(meta) if m[0] <= 12]
    full = set(rng.choice(small, size=min(4, len(small)), replace=False).tolist())
    for i in range(64):
        _oracle_check(meta[i], xs[i].cpu().numpy(), full_solve=i in full)


def test_tuned_inner_paths_in_one_launch(sem):
    """inner = f32_tuned: each problem of one launch takes its order's inner path
    (here N=5 the split FP16 tensor cores, N=7 and N=9 the FP32 CUDA cores), and
    every residual meets the oracle bar; the tuner times both paths."""
    specs = [(3, 5, 1, 2, 1), (2, 7, 1, 1, 1), (2, 9, 2, 1, 1), (4, 5, 1, 1, 2)]
    ctxs, bs, xs, meta = _problems(sem, specs)
    sem.set_inner_path(5, 1)
    sem.set_inner_path(7, 0)
    sem.set_inner_path(9, 0)
    try:
        infos = sem.pcg_solve_batched(ctxs, bs, xs, [1.0] * 4, [0.0] * 4, tol=1e-10, inner="f32_tuned",
                                      inner_tol=1e-4)
        for i, info in enumerate(infos):
            assert info["status"] == 0, (meta[i], info)
            _oracle_check(meta[i], xs[i].cpu().numpy())
        with pytest.raises(sem.SemError):
            sem.set_inner_path(9, 1)  # the split tensor-core path serves N <= 7
        r = sem.tune_inner(ctxs[0], iters=10)
        assert r["path"] in (0, 1) and r["ms_per_iter"][0] > 0 and r["ms_per_iter"][1] > 0, r
        r9 = sem.tune_inner(ctxs[2], iters=10)
        assert r9["path"] == 0 and r9["ms_per_iter"][1] == -1.0, r9
    finally:
        for N in (5, 7, 9):
            sem.set_inner_path(N, 0)
