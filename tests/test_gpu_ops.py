"""GPU parity of setup, sem_ax, sem_dssum and sem_jacobi against the FP64 oracle.

Bars: geometry and FP64 operator max|gpu - ref| / max|ref| <= 1e-12; FP32
operator <= 1e-5 (on the same FP32-rounded input); dssum to rounding of a
sum of at most 8 terms.  Small meshes span several element groups and a
ragged tail; the full 32^3, N=7 deformed mesh is checked on sampled elements
(each recomputed by the oracle on its own one-element mesh) and, for dssum,
against the oracle over the whole field.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_24348_gb300 import inputs

pytestmark = pytest.mark.gpu

TWO_PI = 2 * math.pi
CASES = [(1, (3, 2, 5), 0.1), (2, (3, 2, 5), 0.1), (3, (2, 3, 2), 0.15), (5, (4, 4, 4), 0.0),
         (7, (3, 5, 2), 0.1), (9, (2, 2, 3), 0.1), (15, (2, 1, 2), 0.1)]


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def make(sem, N, nel, perturb, periodic=(1, 1, 1), L=(TWO_PI,) * 3):
    v = inputs.box_vertices(nel, L, perturb=perturb)
    ctx = sem.Ctx(N, nel, L, periodic, vertices=v)
    m = oracle.Mesh(N, nel, v, periodic)
    return ctx, m, v


@pytest.mark.parametrize("N,nel,perturb", CASES)
def test_geometry_and_coords(sem, N, nel, perturb):
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, perturb)
    geo = torch.empty(7 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.geom(geo)
    xyz = torch.empty(3 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.coords(xyz)
    torch.cuda.synchronize()
    g = geo.cpu().numpy().reshape(7, -1)
    for c in range(6):
        assert np.abs(g[c] - m.G[c]).max() <= 1e-13 * np.abs(m.G[:3]).max(), c
    assert rel_err(g[6], m.B) <= 1e-13
    assert rel_err(xyz.cpu().numpy().reshape(3, -1), m.xyz) <= 1e-14
    assert abs(ctx.volume - TWO_PI ** 3) <= 1e-12 * TWO_PI ** 3


@pytest.mark.parametrize("N,nel,perturb", CASES)
@pytest.mark.parametrize("h1,h2", [(1.0, 0.0), (0.01, 1000.0)])
def test_ax_f64_f32(sem, N, nel, perturb, h1, h2):
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, perturb)
    u = inputs.local_uniform_field(ctx.nL, seed=inputs.SEED_FIELD)
    ref = m.ax(u, h1, h2)
    ud = torch.from_numpy(u).to(dev)
    wd = torch.empty_like(ud)
    ctx.ax(ud, wd, h1, h2, "f64")
    assert rel_err(wd.cpu().numpy(), ref) <= 1e-12
    u32 = u.astype(np.float32)
    ref32 = m.ax(u32.astype(np.float64), h1, h2)
    ud32 = torch.from_numpy(u32).to(dev)
    wd32 = torch.empty_like(ud32)
    ctx.ax(ud32, wd32, h1, h2, "f32")
    assert rel_err(wd32.cpu().numpy().astype(np.float64), ref32) <= 1e-5
    assert ctx.device_status() == 0  # no bounded wait of the staged kernel gave up


@pytest.mark.parametrize("dtype,bound", [("bf16_tc", 3e-2), ("f16_tc", 4e-3)])
@pytest.mark.parametrize("N,nel,perturb", [(1, (3, 2, 2), 0.1), (3, (3, 2, 5), 0.1),
                                           (5, (4, 4, 4), 0.1), (7, (3, 5, 2), 0.1),
                                           (9, (2, 2, 3), 0.1)])
def test_ax_tensor_core(sem, dtype, bound, N, nel, perturb):
    """16-bit tensor-core contractions: error of the order of the 16-bit rounding
    (no FP64-level bar), measured on a continuous field."""
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, perturb)
    u = inputs.unique_uniform_field(N, nel, seed=inputs.SEED_FIELD).astype(np.float32)
    for h1, h2 in ((1.0, 0.0), (0.01, 1000.0)):
        ref = m.ax(u.astype(np.float64), h1, h2)
        ud = torch.from_numpy(u).to(dev)
        wd = torch.empty_like(ud)
        ctx.ax(ud, wd, h1, h2, dtype)
        err = rel_err(wd.cpu().numpy().astype(np.float64), ref)
        assert err <= bound, (dtype, N, h1, h2, err)


@pytest.mark.parametrize("dtype", ["f16x2_tc", "bf16x3_tc"])
@pytest.mark.parametrize("N,nel,perturb", [(1, (3, 2, 2), 0.1), (3, (3, 2, 5), 0.1),
                                           (5, (4, 4, 4), 0.1), (7, (3, 5, 2), 0.1)])
def test_ax_tensor_core_split_operands(sem, dtype, N, nel, perturb):
    """Split-operand 16-bit tensor-core contractions reach the FP32 operator's bar
    (<= 1e-5 of the largest output, on the same FP32-rounded input), on a
    discontinuous field and on elements scaled by 2^-40 and 2^40 (the FP16 parts
    are rescaled per element)."""
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, perturb)
    u = inputs.local_uniform_field(ctx.nL, seed=7).astype(np.float32)
    n3 = (N + 1) ** 3
    us = u.reshape(ctx.E, n3).copy()
    us[1] *= np.float32(2.0 ** -40)
    us[2] *= np.float32(2.0 ** 40)
    for x in (u, us.reshape(-1)):
        for h1, h2 in ((1.0, 0.0), (0.01, 1000.0)):
            ref = m.ax(x.astype(np.float64), h1, h2).reshape(ctx.E, n3)
            ud = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
            wd = torch.empty_like(ud)
            ctx.ax(ud, wd, h1, h2, dtype)
            got = wd.cpu().numpy().astype(np.float64).reshape(ctx.E, n3)
            for e in range(ctx.E):  # each element against its own scale
                assert rel_err(got[e], ref[e]) <= 1e-5, (dtype, N, h1, h2, e)


def test_ax_tensor_core_split_rejects_high_order(sem):
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, 8, (1, 1, 1), 0.0)
    u = torch.zeros(ctx.nL, dtype=torch.float32, device=dev)
    with pytest.raises(sem.SemError):
        ctx.ax(u, torch.empty_like(u), 1.0, 0.0, "f16x2_tc")


def test_ax_tensor_core_rejects_high_order(sem):
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, 11, (1, 1, 1), 0.0)
    u = torch.zeros(ctx.nL, dtype=torch.float32, device=dev)
    with pytest.raises(sem.SemError):
        ctx.ax(u, torch.empty_like(u), 1.0, 0.0, "bf16_tc")


def test_autotuner_candidates_keep_parity(sem, tmp_path):
    """Every tile-shape candidate of the FP32 operator gives the same result; the
    tuner's choice is cached per (GPU, N, dtype) and re-applied from the cache."""
    torch, dev = torch_dev()
    for N, nel in ((7, (5, 4, 3)), (5, (4, 4, 5)), (4, (3, 3, 3))):
        ctx, m, _ = make(sem, N, nel, 0.1)
        u32 = inputs.local_uniform_field(ctx.nL, seed=3).astype(np.float32)
        ref = m.ax(u32.astype(np.float64), 0.3, 2.0)
        ud = torch.from_numpy(u32).to(dev)
        for v in range(3):
            sem.set_ax_variant(N, "f32", v)
            wd = torch.empty_like(ud)
            ctx.ax(ud, wd, 0.3, 2.0, "f32")
            assert rel_err(wd.cpu().numpy().astype(np.float64), ref) <= 1e-5, (N, v)
        cache = str(tmp_path / "tune.json")
        r1 = sem.autotune(ctx, "f32", cache=cache)
        assert r1["variant"] in (0, 1, 2) and not r1["cached"] and r1["ms"][0] > 0
        r2 = sem.autotune(ctx, "f32", cache=cache)
        assert r2["cached"] and r2["variant"] == r1["variant"]
        assert ctx.device_status() == 0


def test_autotuner_f64_candidates_keep_parity(sem):
    """Every candidate of the FP64-accurate operator (even N+1: three shapes of the
    float-pair folded kernel, eight of the block-floating-point kernel) is within
    the FP64 bar of the oracle; candidates of one kernel family are identical to
    each other (the grouping of elements into blocks, the staging of u and the
    pairing of instructions do not enter the arithmetic); odd N+1 has one
    candidate."""
    torch, dev = torch_dev()
    for N, nel in ((7, (5, 4, 3)), (5, (4, 4, 5)), (1, (3, 3, 3))):
        ctx, m, _ = make(sem, N, nel, 0.1)
        u = inputs.local_uniform_field(ctx.nL, seed=5)
        ref = m.ax(u, 0.3, 2.0)
        ud = torch.from_numpy(u).to(dev)
        outs = []
        for v in range(11):
            sem.set_ax_variant(N, "f64", v)
            wd = torch.empty_like(ud)
            ctx.ax(ud, wd, 0.3, 2.0, "f64")
            outs.append(wd.cpu().numpy())
            assert rel_err(outs[-1], ref) <= 1e-12, (N, v)
        for v in (1, 2):
            assert np.array_equal(outs[v], outs[0]), (N, v)
        for v in range(4, 11):
            assert np.array_equal(outs[v], outs[3]), (N, v)
        r = sem.autotune(ctx, "f64")
        assert 0 <= r["variant"] <= 10 and len(r["ms"]) == 11 and min(r["ms"]) > 0, r
        sem.set_ax_variant(N, "f64", -1)
        assert ctx.device_status() == 0
    ctx, _, _ = make(sem, 4, (3, 3, 3), 0.1)
    r = sem.autotune(ctx, "f64")
    assert r["variant"] == 0 and r["ms"] == [0.0], r
    sem.set_ax_variant(4, "f64", -1)


def test_ax_host_pointers(sem):
    """Host (numpy) buffers go through the library's staging path."""
    ctx, m, _ = make(sem, 4, (3, 3, 2), 0.1)
    u = inputs.local_uniform_field(ctx.nL, seed=9)
    w = np.zeros_like(u)
    ctx.ax(u, w, 0.5, 2.0, "f64")
    assert rel_err(w, m.ax(u, 0.5, 2.0)) <= 1e-12


@pytest.mark.parametrize("dt", ["f64", "f64_native", "f32", "bf16_tc"])
def test_ax_host_pipeline_equals_device_call(sem, dt):
    """Host buffers run the operator in element chunks with overlapped copies
    (45 elements: 8 chunks of 6, the last one ragged), or, for the FP64-accurate
    operator on pinned buffers, on the mapped host memory directly; every
    element's result is bit-identical to the device-pointer call, for
    host/device mixes too."""
    torch, dev = torch_dev()
    ctx, _, _ = make(sem, 7, (3, 3, 5), 0.1)
    u = inputs.local_uniform_field(ctx.nL, seed=11)
    if dt in ("f32", "bf16_tc"):
        u = u.astype(np.float32)
    ud = torch.from_numpy(u).to(dev)
    wd = torch.empty_like(ud)
    ctx.ax(ud, wd, 0.3, 5.0, dt)
    ref = wd.cpu().numpy()
    uh = torch.from_numpy(u).pin_memory()
    for src, dst in ((uh, torch.empty_like(uh).pin_memory()), (u, np.zeros_like(u)),
                     (uh, torch.empty_like(ud)), (ud, np.zeros_like(u)),
                     (ud, torch.empty_like(uh).pin_memory())):
        ctx.ax(src, dst, 0.3, 5.0, dt)
        got = dst.cpu().numpy() if isinstance(dst, torch.Tensor) else dst
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("N,nel", [(4, (3, 2, 5)), (8, (2, 3, 3))])
def test_ax_f64_on_pinned_host_memory(sem, N, nel):
    """The FP64-accurate operator reads pinned host u and writes pinned host w in
    place (unfolded kernel for odd N+1, folded for even): within the FP64 bar of
    the oracle and bit-identical to the device call."""
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, 0.1)
    u = inputs.local_uniform_field(ctx.nL, seed=12)
    ud = torch.from_numpy(u).to(dev)
    wd = torch.empty_like(ud)
    ctx.ax(ud, wd, 0.7, 3.0, "f64")
    uh = torch.from_numpy(u).pin_memory()
    wh = torch.full_like(uh, float("nan")).pin_memory()
    ctx.ax(uh, wh, 0.7, 3.0, "f64")
    assert np.array_equal(wh.numpy(), wd.cpu().numpy())
    assert rel_err(wh.numpy(), m.ax(u, 0.7, 3.0)) <= 1e-12
    assert ctx.device_status() == 0


def test_ax_empty_input_is_rejected(sem):
    with pytest.raises(sem.SemError):
        sem.Ctx(0, (2, 2, 2))
    with pytest.raises(sem.SemError):
        sem.Ctx(16, (2, 2, 2))
    with pytest.raises(sem.SemError):
        sem.Ctx(3, (0, 2, 2))


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("N,nel", [(1, (3, 1, 2)), (2, (1, 1, 1)), (5, (3, 2, 4)), (8, (2, 3, 1))])
def test_dssum(sem, N, nel, periodic):
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, 0.0, periodic)
    u = inputs.local_uniform_field(ctx.nL, seed=4)
    ref = m.dssum(u)
    ud = torch.from_numpy(u).to(dev)
    ctx.dssum(ud, "f64")
    got = ud.cpu().numpy()
    assert np.abs(got - ref).max() <= 8 * 2.3e-16 * 8
    u32 = torch.from_numpy(u.astype(np.float32)).to(dev)
    ctx.dssum(u32, "f32")
    assert np.abs(u32.cpu().numpy() - ref).max() <= 8 * 1.2e-7 * 8


@pytest.mark.parametrize("N,nel,perturb", [(3, (2, 2, 2), 0.12), (7, (3, 2, 4), 0.1)])
def test_jacobi(sem, N, nel, perturb):
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, perturb)
    for h1, h2 in ((1.0, 0.0), (0.8, 3.0)):
        out = torch.empty(ctx.nL, dtype=torch.float64, device=dev)
        ctx.jacobi(out, h1, h2)
        assert rel_err(out.cpu().numpy(), m.jacobi(h1, h2)) <= 1e-13


def _element_mesh(N, vert, e, nel):
    """One-element oracle mesh of element e of a vertex grid."""
    nx, ny, nz = nel
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    sub = vert[ez:ez + 2, ey:ey + 2, ex:ex + 2, :]
    return oracle.Mesh(N, (1, 1, 1), sub, (0, 0, 0))


def test_ax_full_size_sampled(sem):
    """32^3 elements, N=7, interior vertices perturbed by up to 10% (16.8M nodes):
    both precisions against the oracle on 48 sampled elements (first, last, seeded)."""
    torch, dev = torch_dev()
    N, nel = 7, (32, 32, 32)
    v = inputs.box_vertices(nel, (TWO_PI,) * 3, perturb=0.1)
    ctx = sem.Ctx(N, nel, (TWO_PI,) * 3, (1, 1, 1), vertices=v)
    h1, h2 = 0.01, 1000.0
    u = inputs.unique_uniform_field(N, nel, seed=inputs.SEED_FIELD)
    ud = torch.from_numpy(u).to(dev)
    wd = torch.empty_like(ud)
    ctx.ax(ud, wd, h1, h2, "f64")
    u32 = torch.from_numpy(u.astype(np.float32)).to(dev)
    w32 = torch.empty_like(u32)
    ctx.ax(u32, w32, h1, h2, "f32")
    w = wd.cpu().numpy().reshape(ctx.E, -1)
    w32 = w32.cpu().numpy().reshape(ctx.E, -1)
    u = u.reshape(ctx.E, -1)
    rng = np.random.default_rng(11)
    sample = [0, ctx.E - 1] + list(rng.choice(ctx.E, 46, replace=False))
    err64 = err32 = 0.0
    for e in sample:
        me = _element_mesh(N, v, int(e), nel)
        ref = me.ax(u[e], h1, h2)
        ref32 = me.ax(u[e].astype(np.float32).astype(np.float64), h1, h2)
        err64 = max(err64, np.abs(w[e] - ref).max() / np.abs(ref).max())
        err32 = max(err32, np.abs(w32[e] - ref32).max() / np.abs(ref32).max())
    assert err64 <= 1e-12, err64
    assert err32 <= 1e-5, err32
    assert ctx.device_status() == 0


def test_dssum_full_size(sem):
    torch, dev = torch_dev()
    N, nel = 7, (32, 32, 32)
    ctx = sem.Ctx(N, nel)
    u = inputs.local_uniform_field(ctx.nL, seed=4)
    ud = torch.from_numpy(u).to(dev)
    ctx.dssum(ud, "f64")
    m_idx = inputs.local_to_unique(N, nel)
    # oracle-free closed check: sum of copies by unique index (numpy bincount)
    ref = np.bincount(m_idx, weights=u)[m_idx]
    assert np.abs(ud.cpu().numpy() - ref).max() <= 64 * 2.3e-16


@pytest.mark.parametrize("N,nel", [(1, (3, 4, 2)), (2, (3, 3, 3)), (4, (3, 2, 4)), (7, (4, 3, 3)),
                                   (9, (2, 3, 2)), (15, (2, 2, 1))])
def test_native_f64_operator_matches_oracle(sem, N, nel):
    """The native FP64 operator (the folded even-odd kernel for even N+1, the
    unfolded one otherwise) within 1e-13 of the oracle on a deformed mesh; for
    even N+1 both candidates agree to FP64 rounding and the tuner times both."""
    torch, dev = torch_dev()
    ctx, m, _ = make(sem, N, nel, 0.1)
    u = inputs.local_uniform_field(ctx.nL, seed=21)
    ref = m.ax(u, 0.4, 3.0)
    ud = torch.from_numpy(u).to(dev)
    outs = []
    nvar = 2 if (N + 1) % 2 == 0 else 1
    for v in range(nvar):
        sem.set_ax_variant(N, "f64_native", v)
        wd = torch.empty_like(ud)
        ctx.ax(ud, wd, 0.4, 3.0, "f64_native")
        outs.append(wd.cpu().numpy())
        assert rel_err(outs[-1], ref) <= 1e-13, (N, v, rel_err(outs[-1], ref))
    if nvar == 2:
        assert rel_err(outs[0], outs[1]) <= 1e-14
        r = sem.autotune(ctx, "f64_native")
        assert r["variant"] in (0, 1) and min(r["ms"][:2]) > 0, r
    sem.set_ax_variant(N, "f64_native", -1)
    assert ctx.device_status() == 0
