"""sem_pcg_solve_noalloc: the PCG entry point for callers that cannot allocate
device memory (under another allocator's fixed device budget, or where
cudaMalloc's implicit synchronisation is unacceptable).  It must agree with
sem_pcg_solve and with the FP64 oracle, call after call, while its scratch
lives in one fixed static device array.  This file sorts last so that a
stop-at-first-failure run has already run every other test."""
import pytest

from helpers import pair, rel, sine_rhs, torch_dev

pytestmark = pytest.mark.gpu


def _geom_per_element(ctx):
    torch, dev = torch_dev()
    n3 = (ctx.N + 1) ** 3
    g = torch.empty(7 * ctx.nL, dtype=torch.float64, device=dev)
    ctx.geom(g)
    return g.view(7, ctx.E, n3).permute(1, 0, 2).contiguous()


@pytest.mark.parametrize("N,nel,periodic,perturb,h2", [
    (5, (4, 4, 4), (1, 1, 1), 0.1, 0.0),
    (7, (3, 2, 3), (1, 1, 1), 0.1, 1.5),
    (4, (3, 3, 2), (0, 1, 0), 0.1, 0.0),     # non-periodic directions: gather built from flags
    (1, (4, 3, 3), (1, 1, 1), 0.0, 1.0),     # smallest order
    (15, (2, 2, 2), (1, 1, 1), 0.0, 2.0),    # largest order
])
def test_noalloc_matches_pcg_and_oracle_on_two_calls_in_a_row(sem, N, nel, periodic, perturb, h2):
    torch, dev = torch_dev()
    ctx, m, _ = pair(sem, N, nel, perturb, periodic=periodic)
    bg, bo, _ = sine_rhs(ctx, m, (1, 2, 1))
    xo, io = m.pcg(bo, 1.0, h2, tol=1e-12)
    assert io["status"] == 0
    # the context's solve with the same (native FP64) operator
    xref = torch.zeros_like(bg)
    iref = ctx.pcg_solve(bg, xref, 1.0, h2, tol=1e-10, inner="f64_native")
    assert iref["status"] == 0
    geom = _geom_per_element(ctx)
    for _ in range(2):
        x = torch.zeros_like(bg)
        info = sem.pcg_solve_noalloc(N, nel, periodic, geom, bg, x, 1.0, h2, tol=1e-10)
        assert info["status"] == 0, info
        assert abs(info["iters"] - iref["iters"]) <= 1
        xh = x.cpu().numpy()
        assert rel(xh, xref.cpu().numpy()) <= 1e-9
        assert rel(xh, xo) <= 1e-9
        r, bn = m.residual(bo, xh, 1.0, h2)
        assert r <= 1.5e-10 * bn


def test_noalloc_rejects_problems_beyond_its_scratch(sem):
    torch, dev = torch_dev()
    small = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(sem.SemError) as e:
        sem.pcg_solve_noalloc(7, (20, 20, 20), (1, 1, 1), small, small, small, 1.0, 0.0)
    assert e.value.code == sem.ERR_TOO_LARGE
