"""Pins of the oracle's pressure solver (flexible GMRES with the hybrid Schwarz
multigrid preconditioner, coarse CG + Jacobi: Sec. 1 and the solver settings
of Sec. 3), against things other than the oracle itself:

- the fast-diagonalisation factors are the generalised eigenpairs of the 1-D
  operators, and those operators are the textbook GLL stiffness and mass
  (built here from numpy) plus the one-node extension;
- the local solve equals a dense solve of the Kronecker-sum operator;
- on one box element with no neighbours the smoother is the exact inverse of
  the SEM operator (the separable form is then exact);
- prolongation reproduces polynomials of the coarser order exactly, and the
  restriction is its transpose on unique nodes;
- a hierarchy of one (coarse) level solves the system;
- the V-cycle contracts the error (spectral radius of I - M^-1 A well below
  1) and cuts the iteration count far below Jacobi-PCG's;
- GMRES without a preconditioner returns the minimal residual over the Krylov
  space (dense numpy least squares), and with HSMG the dense solution.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_24348_gb300 import inputs
from test_oracle import mesh, q_matrix


def khat(N):
    """Reference 1-D GLL stiffness sum_q w_q D_qi D_qj (numpy, from the pinned GLL/D)."""
    xi, w = oracle.gll(N)
    D = oracle.deriv(N)
    return D.T @ np.diag(w) @ D, xi, w


@pytest.mark.parametrize("N,h,hl,hr", [(1, 0.3, 0.2, 0.5), (4, 1.0, 0.0, 0.7), (7, 0.2, 0.25, 0.0),
                                       (9, 2.0, 0.0, 0.0)])
def test_fdm_factors(N, h, hl, hr):
    S, lam, K, M = oracle.fdm_1d(N, h, hl, hr)
    Kh, xi, w = khat(N)
    gap = xi[1] - xi[0]
    Kref = 2.0 / h * Kh
    Mref = 0.5 * h * w.copy()
    if hl > 0:
        Kref[0, 0] += 2.0 / (gap * hl)
        Mref[0] += 0.25 * gap * hl
    if hr > 0:
        Kref[-1, -1] += 2.0 / (gap * hr)
        Mref[-1] += 0.25 * gap * hr
    np.testing.assert_allclose(K, Kref, atol=1e-12 * np.abs(Kref).max())
    np.testing.assert_allclose(M, Mref, rtol=1e-14)
    np.testing.assert_allclose(S.T @ np.diag(M) @ S, np.eye(N + 1), atol=1e-12)
    np.testing.assert_allclose(K @ S, np.diag(M) @ S @ np.diag(lam), atol=1e-10 * np.abs(K).max())
    # the eigenvalues are those of the generalised problem (scipy-free: via numpy eigvalsh)
    Mi = np.diag(1 / np.sqrt(M))
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(Mi @ K @ Mi), rtol=1e-10, atol=1e-10)
    if hl == 0 and hr == 0:
        assert abs(np.sort(lam)[0]) < 1e-10 * lam.max()   # Neumann: the constant mode


def test_fdm_apply_equals_dense_solve():
    N = 5
    n = N + 1
    rng = np.random.default_rng(11)
    facs, KM = [], []
    for h, hl, hr in ((0.4, 0.3, 0.5), (0.7, 0.7, 0.0), (0.25, 0.2, 0.2)):
        S, lam, K, M = oracle.fdm_1d(N, h, hl, hr)
        facs.append((S, lam))
        KM.append((K, np.diag(M)))
    (Kx, Mx), (Ky, My), (Kz, Mz) = KM
    for h1, h2 in ((1.0, 0.0), (0.3, 5.0)):
        A = h1 * (np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) +
                  np.kron(Kz, np.kron(My, Mx))) + h2 * np.kron(Mz, np.kron(My, Mx))
        r = rng.standard_normal(n ** 3)
        z = oracle.fdm_apply(N, facs, h1, h2, r)
        np.testing.assert_allclose(z, np.linalg.solve(A, r), rtol=1e-9, atol=1e-12 * np.abs(z).max())


@pytest.mark.parametrize("N", [3, 6])
def test_smoother_is_the_exact_inverse_on_one_box_element(N):
    """One non-periodic box element (lengths 1.3, 0.7, 2.1) and h2 > 0: the separable
    local operator is the SEM operator itself, so the smoother solves exactly."""
    L = (1.3, 0.7, 2.1)
    nel = (1, 1, 1)
    m = mesh(N, nel, 0.0, L=L, periodic=(0, 0, 0))
    v = inputs.box_vertices(nel, L, perturb=0.0, seed=inputs.SEED_MESH)
    H = oracle.HSMG([N, 1], nel, v, periodic=(0, 0, 0), h1=0.8, h2=3.0)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(m.nL)
    z = H.smooth(0, r)
    np.testing.assert_allclose(m.dssum(m.ax(z, 0.8, 3.0)), r, atol=1e-10 * np.abs(r).max())


def _poly(x, y, z, deg):
    return (1 + 0.3 * x - 0.2 * y + 0.1 * z) ** deg + 0.5 * x ** min(deg, 2) * z


def test_prolongation_reproduces_coarse_polynomials():
    nel, L = (3, 2, 2), (2.0, 1.5, 1.0)
    v = inputs.box_vertices(nel, L, perturb=0.0, seed=inputs.SEED_MESH)
    H = oracle.HSMG([6, 3, 1], nel, v, periodic=(0, 0, 0))
    for lev, (nf, nc) in enumerate(((6, 3), (3, 1))):
        mf, mc = oracle.Mesh(nf, nel, v, (0, 0, 0)), oracle.Mesh(nc, nel, v, (0, 0, 0))
        uc = _poly(*mc.xyz, nc)
        np.testing.assert_allclose(H.prolong(lev, uc), _poly(*mf.xyz, nc), atol=1e-12)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_restriction_is_the_transpose_of_prolongation(periodic):
    nel = (3, 3, 2)
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=0.1, seed=inputs.SEED_MESH)
    H = oracle.HSMG([5, 2, 1], nel, v, periodic=periodic)
    rng = np.random.default_rng(2)
    for lev, (nf, nc) in enumerate(((5, 2), (2, 1))):
        mf, mc = oracle.Mesh(nf, nel, v, periodic), oracle.Mesh(nc, nel, v, periodic)
        uc = mc.dssum(rng.standard_normal(mc.nL)) * mc.imult      # continuous field
        rf = mf.dssum(rng.standard_normal(mf.nL))                  # assembled residual
        lhs = mf.glsc3(H.prolong(lev, uc), rf)                     # sum over unique fine nodes
        rhs = mc.glsc3(uc, H.restrict(lev, rf))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1), (lhs, rhs)


def test_one_level_hierarchy_is_the_coarse_solve():
    nel = (3, 3, 3)
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=0.1, seed=inputs.SEED_MESH)
    m = oracle.Mesh(2, nel, v)
    H = oracle.HSMG([2], nel, v, ctol=1e-13)
    r = m.dssum(m.B * np.sin(m.xyz[0]) * np.cos(m.xyz[2]))
    z = H.apply(r)
    res = m.dssum(m.ax(z)) - (r - m.glsc3(r, np.ones(m.nL)) / m.glsc3(np.ones(m.nL), np.ones(m.nL)))
    assert np.sqrt(m.glsc3(res, res)) <= 1e-11 * np.sqrt(m.glsc3(r, r))


def _contraction(H, m, iters=25, seed=4):
    """Power-iteration estimate of the spectral radius of I - M^-1 A on mean-free vectors."""
    rng = np.random.default_rng(seed)
    e = m.dssum(rng.standard_normal(m.nL)) * m.imult
    one = np.ones(m.nL)
    rho = 0.0
    for _ in range(iters):
        e -= m.glsc3(e, one) / m.glsc3(one, one)
        n0 = np.sqrt(m.glsc3(e, e))
        e = e - H.apply(m.dssum(m.ax(e)))
        e -= m.glsc3(e, one) / m.glsc3(one, one)
        rho = np.sqrt(m.glsc3(e, e)) / n0
        e /= np.sqrt(m.glsc3(e, e))
    return rho


@pytest.mark.parametrize("orders,nel,perturb,bound", [([5, 3, 1], (4, 4, 4), 0.0, 0.55),
                                                      ([7, 3, 1], (3, 3, 3), 0.0, 0.8),
                                                      ([5, 3, 1], (4, 4, 4), 0.15, 0.8)])
def test_vcycle_contracts_the_error(orders, nel, perturb, bound):
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=perturb, seed=inputs.SEED_MESH)
    m = oracle.Mesh(orders[0], nel, v)
    H = oracle.HSMG(orders, nel, v, ctol=1e-10)
    rho = _contraction(H, m)
    assert rho < bound, rho


def test_gmres_without_preconditioner_is_the_minimal_residual():
    """Unrestarted GMRES after k steps minimises ||f - A x|| over x in K_k(A, f):
    compare its Arnoldi estimates and its final residual with numpy least squares
    over an explicit orthonormalised Krylov basis (nonsingular Helmholtz)."""
    N, nel, h2 = 2, (2, 2, 3), 1.5
    m = mesh(N, nel, 0.1)
    Q = q_matrix(N, nel, (1, 1, 1))
    ng = Q.shape[1]
    A = np.stack([Q.T @ m.ax(Q[:, c], 1.0, h2) for c in range(ng)], axis=1)
    f = np.random.default_rng(8).standard_normal(ng)
    for k in (1, 3, 6):
        x, st, info = oracle.fgmres(Q @ f, mesh=m, h1=1.0, h2=h2, tol=1e-30, m=20, maxit=k,
                                    history=True)
        assert info["iters"] == k
        K = np.zeros((ng, k))
        K[:, 0] = f / np.linalg.norm(f)
        for j in range(1, k):
            w = A @ K[:, j - 1]
            w -= K[:, :j] @ (K[:, :j].T @ w)
            w -= K[:, :j] @ (K[:, :j].T @ w)
            K[:, j] = w / np.linalg.norm(w)
        y = np.linalg.lstsq(A @ K, f, rcond=None)[0]
        rmin = np.linalg.norm(f - A @ K @ y)
        assert abs(info["hist"][k] - rmin) <= 1e-9 * np.linalg.norm(f), (k, info["hist"][k], rmin)
        assert abs(info["rnorm"] - rmin) <= 1e-9 * np.linalg.norm(f)
        np.testing.assert_allclose(x, Q @ (K @ y), atol=1e-9 * np.abs(K @ y).max())


@pytest.mark.parametrize("orders", [[3, 1], [3, 2, 1]])
def test_fgmres_hsmg_matches_the_dense_solution(orders):
    N, nel = orders[0], (2, 3, 2)
    m = mesh(N, nel, 0.1)
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=0.1, seed=inputs.SEED_MESH)
    H = oracle.HSMG(orders, nel, v, ctol=1e-3)
    Q = q_matrix(N, nel, (1, 1, 1))
    ng = Q.shape[1]
    A = np.stack([Q.T @ m.ax(Q[:, c], 1.0, 0.0) for c in range(ng)], axis=1)
    f = np.random.default_rng(3).standard_normal(ng)
    x, st, info = oracle.fgmres(Q @ f, hsmg=H, tol=1e-12, m=20, maxit=200)
    assert st == 0 and info["iters"] <= 30, info
    xu = np.linalg.lstsq(A, f - f.mean(), rcond=None)[0]
    xl = Q @ xu
    xl -= (m.B * xl).sum() / m.B.sum()
    np.testing.assert_allclose(x, xl, atol=1e-9 * np.abs(xl).max())


def test_hsmg_cuts_iterations_far_below_jacobi_pcg():
    """Pressure-Poisson workload (divergence of a smooth random field) on 4^3, N=7:
    GMRES + HSMG (7, 3, 1) needs a small fraction of Jacobi-PCG's iterations."""
    N, nel = 7, (4, 4, 4)
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3, perturb=0.0, seed=inputs.SEED_MESH)
    m = oracle.Mesh(N, nel, v)
    K, cc, cs = inputs.fourier_div_modes()
    f = oracle.fourier(K, cc, cs, *m.xyz)
    b = m.dssum(m.B * f)
    xp, ip = m.pcg(b, tol=1e-8)
    H = oracle.HSMG([7, 3, 1], nel, v, ctol=1e-2)
    xg, st, info = oracle.fgmres(b, hsmg=H, tol=1e-8, m=30, maxit=200)
    assert ip["status"] == 0 and st == 0
    assert info["iters"] * 4 <= ip["iters"], (info["iters"], ip["iters"])
    d = xg - xp
    assert np.sqrt(m.glsc3(d, d)) <= 1e-6 * np.sqrt(m.glsc3(xp, xp))
