"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: closed
forms, library routines on special cases (numpy's Legendre tools and dense
linear algebra), brute force on tiny inputs built independently here, and
invariants of the method.  None of it needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_24348_gb300 import inputs

NOTGPU = pytest.mark.filterwarnings("ignore")


# ----------------------------------------------------------------------------
# helpers built independently of the oracle
# ----------------------------------------------------------------------------

def lagrange_basis(nodes, x):
    """l_j(x_q) for the nodes, by the product formula (test-side)."""
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                L[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return L


def lagrange_deriv(nodes, x):
    """l_j'(x_q) via numpy polynomial objects."""
    n = len(nodes)
    out = np.zeros((len(x), n))
    for j in range(n):
        others = [nodes[k] for k in range(n) if k != j]
        p = np.polynomial.Polynomial.fromroots(others)
        p = p / p(nodes[j])
        out[:, j] = p.deriv()(x)
    return out


def q_matrix(N, nel, periodic):
    """Dense scatter matrix Q (local x unique) from the index layout."""
    g = inputs.local_to_unique(N, nel, periodic)
    ng = int(np.prod(inputs.unique_counts(N, nel, periodic)))
    Q = np.zeros((g.size, ng))
    Q[np.arange(g.size), g] = 1.0
    return Q


def mesh(N, nel, perturb=0.0, L=(2 * math.pi,) * 3, periodic=(1, 1, 1)):
    v = inputs.box_vertices(nel, L, perturb=perturb, seed=inputs.SEED_MESH)
    return oracle.Mesh(N, nel, v, periodic)


# ----------------------------------------------------------------------------
# GLL / GL / D / interpolation
# ----------------------------------------------------------------------------

def test_gll_closed_forms():
    xi, w = oracle.gll(1)
    np.testing.assert_allclose(xi, [-1, 1], atol=0)
    np.testing.assert_allclose(w, [1, 1], rtol=1e-15)
    xi, w = oracle.gll(2)
    np.testing.assert_allclose(xi, [-1, 0, 1], atol=1e-16)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    xi, w = oracle.gll(3)
    s = 1 / math.sqrt(5)
    np.testing.assert_allclose(xi, [-1, -s, s, 1], rtol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)


@pytest.mark.parametrize("N", list(range(2, 16)))
def test_gll_interior_are_roots_of_legendre_derivative(N):
    xi, w = oracle.gll(N)
    roots = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
    np.testing.assert_allclose(xi[1:-1], roots, atol=2e-14)
    np.testing.assert_allclose(xi, -xi[::-1], atol=0)
    np.testing.assert_allclose(w, w[::-1], rtol=0)


@pytest.mark.parametrize("N", list(range(1, 16)))
def test_gll_quadrature_exact_to_2N_minus_1(N):
    xi, w = oracle.gll(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs((w * xi ** k).sum() - exact) < 1e-14, (N, k)
    k = 2 * N
    assert abs((w * xi ** k).sum() - 2.0 / (k + 1)) > 1e-9  # GLL, not Gauss


@pytest.mark.parametrize("M", [1, 2, 5, 9, 12, 15, 24])
def test_gl_matches_numpy_leggauss(M):
    eta, w = oracle.gl(M)
    x, wx = np.polynomial.legendre.leggauss(M)
    np.testing.assert_allclose(eta, x, atol=1e-15)
    np.testing.assert_allclose(w, wx, rtol=5e-13)


@pytest.mark.parametrize("N", list(range(1, 16)))
def test_derivative_matrix(N):
    xi, _ = oracle.gll(N)
    D = oracle.deriv(N)
    # exact on monomials up to degree N
    for k in range(0, N + 1):
        d = D @ xi ** k
        ref = k * xi ** (k - 1) if k else np.zeros_like(xi)
        assert np.abs(d - ref).max() < 1e-12 * max(1, N * N), (N, k)
    np.testing.assert_allclose(D @ np.ones(N + 1), 0, atol=1e-13)
    # centro-symmetry D_{N-i,N-j} = -D_ij
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-12)
    # corner closed forms
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-11
    assert abs(D[N, N] - N * (N + 1) / 4) < 1e-11
    # against an independent construction of l_j'(xi_i)
    np.testing.assert_allclose(D, lagrange_deriv(xi, xi), atol=1e-10 * N * N)


@pytest.mark.parametrize("N", [1, 4, 7, 9])
def test_interp_matrix(N):
    xi, _ = oracle.gll(N)
    x = np.linspace(-1, 1, 13) * 0.97
    J = oracle.interp(N, x)
    np.testing.assert_allclose(J, lagrange_basis(xi, x), atol=1e-14)
    for k in range(N + 1):
        np.testing.assert_allclose(J @ xi ** k, x ** k, atol=1e-13)
    np.testing.assert_allclose(oracle.interp(N, xi), np.eye(N + 1), atol=1e-15)


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------

def test_geometry_undeformed_closed_form():
    N, nel, L = 4, (3, 2, 5), (1.0, 2.0, 3.0)
    m = mesh(N, nel, 0.0, L)
    hx, hy, hz = L[0] / nel[0], L[1] / nel[1], L[2] / nel[2]
    xi, w = oracle.gll(N)
    n = N + 1
    W = (w[None, None, :] * w[None, :, None] * w[:, None, None]).reshape(-1)
    E = m.E
    G = m.G.reshape(6, E, -1)
    np.testing.assert_allclose(G[0], np.broadcast_to(W * hy * hz / (2 * hx), (E, n ** 3)), rtol=1e-13)
    np.testing.assert_allclose(G[1], np.broadcast_to(W * hx * hz / (2 * hy), (E, n ** 3)), rtol=1e-13)
    np.testing.assert_allclose(G[2], np.broadcast_to(W * hx * hy / (2 * hz), (E, n ** 3)), rtol=1e-13)
    assert np.abs(G[3:]).max() < 1e-15
    np.testing.assert_allclose(m.B.reshape(E, -1), np.broadcast_to(W * hx * hy * hz / 8, (E, n ** 3)),
                               rtol=1e-13)
    # node coordinates of element (ex,ey,ez) = (1,1,2)
    e = 1 + nel[0] * (1 + nel[1] * 2)
    X = m.xyz.reshape(3, E, n, n, n)[:, e]
    np.testing.assert_allclose(X[0], np.broadcast_to(hx * (1 + (xi + 1) / 2), (n, n, n)), rtol=1e-14)
    np.testing.assert_allclose(X[1], np.broadcast_to((hy * (1 + (xi + 1) / 2))[:, None], (n, n, n)),
                               rtol=1e-14)
    np.testing.assert_allclose(X[2], np.broadcast_to((hz * (2 + (xi + 1) / 2))[:, None, None],
                                                     (n, n, n)), rtol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 7])
def test_geometry_deformed_volume_and_metrics(N):
    nel = (4, 3, 5)
    m = mesh(N, nel, 0.1)
    assert abs(m.B.sum() - (2 * math.pi) ** 3) < 1e-12 * (2 * math.pi) ** 3
    assert m.B.min() > 0
    # the coordinate functions are degree 1 per direction, so D and J^-1
    # reproduce their gradient exactly: d x_c / d x_d = delta_cd
    n, E = N + 1, m.E
    D = m.D
    for c in range(3):
        X = m.xyz[c].reshape(E, n, n, n)
        dr = np.einsum("il,ekjl->ekji", D, X).reshape(-1)
        ds = np.einsum("jl,ekli->ekji", D, X).reshape(-1)
        dt = np.einsum("kl,elji->ekji", D, X).reshape(-1)
        for d in range(3):
            g = m.jinv[0 * 3 + d] * dr + m.jinv[1 * 3 + d] * ds + m.jinv[2 * 3 + d] * dt
            np.testing.assert_allclose(g, 1.0 if c == d else 0.0, atol=1e-12)
    # G from J^-1 (independent assembly)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for g, (a, b) in enumerate(pairs):
        s = sum(m.jinv[a * 3 + c] * m.jinv[b * 3 + c] for c in range(3))
        np.testing.assert_allclose(m.G[g], m.B * s, rtol=1e-12, atol=1e-14)


def test_geometry_rejects_inverted_element():
    v = inputs.box_vertices((2, 2, 2), (1, 1, 1))
    v[1, 1, 1, 0] = 1.2  # centre vertex pushed past the far boundary plane
    with pytest.raises(ValueError):
        oracle.Mesh(3, (2, 2, 2), v)


# ----------------------------------------------------------------------------
# Element operator
# ----------------------------------------------------------------------------

def test_ax_affine_element_equals_kronecker_matrix():
    N, h1, h2 = 4, 0.7, 2.5
    L = (1.3, 0.8, 2.1)
    m = mesh(N, (1, 1, 1), 0.0, L, periodic=(0, 0, 0))
    xi, w = oracle.gll(N)
    Dl = lagrange_deriv(xi, xi)
    K1 = Dl.T @ np.diag(w) @ Dl
    M1 = np.diag(w)
    hx, hy, hz = L
    # index order u[k][j][i] -> kron(z, y, x)
    A = h1 * (hy * hz / (2 * hx) * np.kron(M1, np.kron(M1, K1))
              + hx * hz / (2 * hy) * np.kron(M1, np.kron(K1, M1))
              + hx * hy / (2 * hz) * np.kron(K1, np.kron(M1, M1))) \
        + h2 * hx * hy * hz / 8 * np.kron(M1, np.kron(M1, M1))
    n3 = (N + 1) ** 3
    cols = np.stack([m.ax(np.eye(n3)[c], h1, h2) for c in range(n3)], axis=1)
    np.testing.assert_allclose(cols, A, atol=1e-12 * np.abs(A).max())


def test_ax_deformed_equals_quadrature_bilinear_form():
    """v^T A u = sum_q w_q |J_q| (h1 grad u . grad v + h2 u v) with grad from J^-1."""
    N, nel, h1, h2 = 3, (3, 3, 3), 1.3, 0.4
    m = mesh(N, nel, 0.15)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(m.nL)
    v = rng.standard_normal(m.nL)
    n, E = N + 1, m.E

    def grad(f):
        F = f.reshape(E, n, n, n)
        dr = np.einsum("il,ekjl->ekji", m.D, F).reshape(-1)
        ds = np.einsum("jl,ekli->ekji", m.D, F).reshape(-1)
        dt = np.einsum("kl,elji->ekji", m.D, F).reshape(-1)
        return [m.jinv[0 * 3 + c] * dr + m.jinv[1 * 3 + c] * ds + m.jinv[2 * 3 + c] * dt
                for c in range(3)]

    gu, gv = grad(u), grad(v)
    ref = (m.B * (h1 * sum(gu[c] * gv[c] for c in range(3)) + h2 * u * v)).sum()
    got = v @ m.ax(u, h1, h2)
    assert abs(got - ref) < 1e-12 * abs(ref)


def test_assembled_operator_symmetric_psd_with_constant_nullspace():
    N, nel = 3, (2, 2, 2)
    m = mesh(N, nel, 0.1)
    Q = q_matrix(N, nel, (1, 1, 1))
    ng = Q.shape[1]
    A = np.stack([Q.T @ m.ax(Q[:, c], 1.0, 0.0) for c in range(ng)], axis=1)
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 1  # only the constants
    one = np.ones(m.nL)
    assert np.abs(m.dssum(m.ax(one, 1.0, 0.0))).max() < 1e-12 * np.abs(A).max()


# ----------------------------------------------------------------------------
# dssum / multiplicity / Jacobi
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("N", [1, 2, 5])
def test_dssum_is_QQt_and_multiplicity(N, periodic):
    nel = (3, 1, 2)
    m = mesh(N, nel, 0.0, periodic=periodic)
    Q = q_matrix(N, nel, periodic)
    u = np.random.default_rng(1).standard_normal(m.nL)
    np.testing.assert_allclose(m.dssum(u), Q @ (Q.T @ u), rtol=1e-14, atol=1e-14)
    # multiplicity closed form: product over directions of (2 at shared planes, else 1)
    n = N + 1
    mult = np.ones((m.E, n, n, n))
    idx = np.arange(m.E)
    ex, ey, ez = idx % nel[0], (idx // nel[0]) % nel[1], idx // (nel[0] * nel[1])
    for d, (e_d, axis) in enumerate(((ex, 3), (ey, 2), (ez, 1))):
        for end, l in ((0, 0), (1, N)):
            shared = np.ones(m.E, bool) if periodic[d] else (e_d > 0 if end == 0 else e_d < nel[d] - 1)
            sl = [slice(None)] * 4
            sl[axis] = l
            sl[0] = shared
            mult[tuple(sl)] *= 2
    np.testing.assert_array_equal(m.mult.reshape(m.E, n, n, n), mult)
    # continuous field is invariant under dssum(u/mult)
    uc = inputs.unique_uniform_field(N, nel, periodic, seed=5)
    np.testing.assert_allclose(m.dssum(uc / m.mult), uc, rtol=1e-14)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("N", [1, 3, 6])
def test_glsc3_with_inverse_multiplicity_is_the_assembled_product(N, periodic):
    """<a, b> = sum_local a b / mult equals sum over unique nodes a_g b_g for
    continuous fields (the solver's norm, Sec. 2 glsc3).  The unique values
    and their multiplicities come from the index layout here, not from the
    oracle's dssum, so a dropped, inverted or squared weight fails."""
    nel = (3, 2, 2)
    m = mesh(N, nel, 0.1, periodic=periodic)
    g = inputs.local_to_unique(N, nel, periodic)
    ng = int(np.prod(inputs.unique_counts(N, nel, periodic)))
    ag = np.random.default_rng(11).uniform(-1, 1, ng)
    bg = np.random.default_rng(12).uniform(-1, 1, ng)
    a, b = ag[g], bg[g]
    exact = float(ag @ bg)
    assert abs(m.glsc3(a, b) - exact) <= 1e-14 * np.abs(ag * bg).sum()
    # the weights themselves: 1 / (number of local copies of each unique node)
    counts = np.bincount(g, minlength=ng).astype(np.float64)
    np.testing.assert_array_equal(m.imult, 1.0 / counts[g])
    # explicit weights: a plain triple product
    c = np.random.default_rng(13).uniform(0.5, 2.0, m.nL)
    assert abs(m.glsc3(a, b, c) - float(np.sum(a * b * c))) <= 1e-14 * np.abs(a * b * c).sum()
    # the norm of the constant is the square root of the unique-node count
    one = np.ones(m.nL)
    assert abs(m.glsc3(one, one) - ng) <= 1e-12 * ng


@pytest.mark.parametrize("k", [(1, 0, 0), (0, -3, 2), (2, 5, -1)])
def test_fourier_single_modes_match_numpy(k):
    """One mode k with coefficients (cc, cs): cc cos(k.x) + cs sin(k.x), evaluated
    with numpy's cos/sin directly; two modes add."""
    rng = np.random.default_rng(7)
    x, y, z = (rng.uniform(-7, 7, 500) for _ in range(3))
    K = np.array([k], dtype=np.int64)
    ph = k[0] * x + k[1] * y + k[2] * z
    np.testing.assert_allclose(oracle.fourier(K, [0.7], [0.0], x, y, z), 0.7 * np.cos(ph),
                               rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.fourier(K, [0.0], [-1.3], x, y, z), -1.3 * np.sin(ph),
                               rtol=0, atol=1e-13)
    K2 = np.array([k, (1, 1, 1)], dtype=np.int64)
    ph2 = x + y + z
    np.testing.assert_allclose(oracle.fourier(K2, [0.5, 0.25], [0.0, 2.0], x, y, z),
                               0.5 * np.cos(ph) + 0.25 * np.cos(ph2) + 2.0 * np.sin(ph2),
                               rtol=0, atol=1e-12)


def test_jacobi_equals_assembled_diagonal():
    N, nel, h1, h2 = 3, (2, 2, 2), 0.8, 3.0
    m = mesh(N, nel, 0.12)
    Q = q_matrix(N, nel, (1, 1, 1))
    ng = Q.shape[1]
    diag = np.array([Q[:, c] @ m.ax(Q[:, c], h1, h2) for c in range(ng)])
    np.testing.assert_allclose(1.0 / m.jacobi(h1, h2), Q @ diag, rtol=1e-13)


# ----------------------------------------------------------------------------
# PCG
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("h2", [0.0, 2.0])
def test_pcg_matches_dense_solve(h2):
    N, nel = 3, (2, 3, 2)
    m = mesh(N, nel, 0.1)
    Q = q_matrix(N, nel, (1, 1, 1))
    ng = Q.shape[1]
    A = np.stack([Q.T @ m.ax(Q[:, c], 1.0, h2) for c in range(ng)], axis=1)
    f = np.random.default_rng(3).standard_normal(ng)
    b_loc = Q @ f                              # assembled vector, stored locally
    x, info = m.pcg(b_loc, 1.0, h2, tol=1e-13)
    assert info["status"] == 0
    if h2 == 0:
        fm = f - f.mean()
        xu = np.linalg.lstsq(A, fm, rcond=None)[0]
        xl = Q @ xu
        xl -= (m.B * xl).sum() / m.B.sum()
    else:
        xl = Q @ np.linalg.solve(A, f)
    np.testing.assert_allclose(x, xl, atol=1e-10 * np.abs(xl).max())
    r, bn = m.residual(b_loc, x, 1.0, h2)
    assert r <= 1e-13 * bn * 1.0001


def test_pcg_status_codes():
    m = mesh(3, (2, 2, 2), 0.1)
    b = m.dssum(m.B * np.sin(m.xyz[0]))
    x, info = m.pcg(b, tol=1e-14, maxit=2)
    assert info["status"] == oracle.ERR_NOT_CONVERGED and info["iters"] == 2
    bad = b.copy(); bad[5] = np.nan
    x, info = m.pcg(bad, tol=1e-10)
    assert info["status"] == oracle.ERR_BREAKDOWN
    x, info = m.pcg(np.zeros(m.nL), tol=1e-10)
    assert info["status"] == 0 and info["iters"] == 0 and not np.any(x)


def test_manufactured_solution_spectral_convergence():
    """u* = sin x sin y sin z on the periodic cube: max error decays spectrally in N."""
    errs = []
    for N in (3, 5, 7, 9):
        m = mesh(N, (2, 2, 2), 0.0)
        x, y, z = m.xyz
        us = np.sin(x) * np.sin(y) * np.sin(z)
        b = m.dssum(m.B * 3 * us)
        sol, info = m.pcg(b, tol=1e-12)
        assert info["status"] == 0
        errs.append(np.abs(sol - us).max())
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1] * 0.1), errs   # > 10x per +2 in N
    assert errs[-1] < 1e-6


# ----------------------------------------------------------------------------
# Convection, diagnostics, TGV stepper
# ----------------------------------------------------------------------------

def test_convection_exact_on_affine_element_against_brute_force():
    """On an affine element and polynomial fields the 3/2-rule integral is exact:
    compare with a (2M)-point Gauss rule built here from numpy."""
    N = 4
    L = (1.3, 0.9, 1.7)
    m = mesh(N, (1, 1, 1), 0.0, L, periodic=(0, 0, 0))
    n = N + 1
    rng = np.random.default_rng(7)
    U = [rng.standard_normal(n ** 3) for _ in range(3)]
    C = m.convect(*U)
    xi, _ = oracle.gll(N)
    M = oracle.dealias_m(N)
    x, wq = np.polynomial.legendre.leggauss(2 * M)
    Lb = lagrange_basis(xi, x)          # (Q, n)
    Ld = lagrange_deriv(xi, x)
    jac = np.array(L) / 2               # dx/dr per direction
    def ev(f, bx, by, bz):
        F = f.reshape(n, n, n)          # [k][j][i]
        return np.einsum("ai,bj,ck,kji->cba", bx, by, bz, F)
    uq = [ev(U[d], Lb, Lb, Lb) for d in range(3)]
    W = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * np.prod(jac)
    for c in range(3):
        grads = [ev(U[c], Ld, Lb, Lb) / jac[0], ev(U[c], Lb, Ld, Lb) / jac[1],
                 ev(U[c], Lb, Lb, Ld) / jac[2]]
        f = W * sum(uq[d] * grads[d] for d in range(3))
        ref = np.einsum("ai,bj,ck,cba->kji", Lb, Lb, Lb, f).reshape(-1)
        np.testing.assert_allclose(C[c], ref, atol=1e-12 * np.abs(ref).max())


def test_convection_of_2d_taylor_green():
    """(u.grad)u of the 2-D Taylor-Green field is (sin 2x, sin 2y, 0)/2."""
    m = mesh(7, (6, 6, 2), 0.0)
    x, y, z = m.xyz
    u, v, w, _ = inputs.tg2d_exact(x, y, z, 0.0, 0.0)
    C = m.convect(u, v, w)
    scale = np.abs(m.B).max()
    np.testing.assert_allclose(C[0], m.B * 0.5 * np.sin(2 * x), atol=2e-6 * scale)
    np.testing.assert_allclose(C[1], m.B * 0.5 * np.sin(2 * y), atol=2e-6 * scale)
    assert np.abs(C[2]).max() < 1e-13 * scale


def test_tgv_initial_energy_and_enstrophy():
    m = mesh(7, (8, 8, 8), 0.0)
    x, y, z = m.xyz
    u, v, w, _ = inputs.tgv_initial(x, y, z)
    ke, en = m.diag(u, v, w, (2 * math.pi) ** 3)
    assert abs(ke - 0.125) < 1e-9
    assert abs(en - 0.375) < 1e-6


def _tg_error(nu, dt, T, N=9, nel=(4, 4, 1)):
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3)
    m = oracle.Mesh(N, nel, v)
    x, y, z = m.xyz
    tgv = oracle.TGV(N, nel, v, (2 * math.pi,) * 3, nu, dt, tol_v=1e-13, tol_p=1e-13,
                     abs_tol=False)
    # exact history for a third-order start
    for lev in (2, 1, 0):
        u, vv, w, p = inputs.tg2d_exact(x, y, z, -lev * dt, nu)
        tgv.set(u, vv, w, p if lev == 0 else None, level=lev, step=2, t=0.0)
    nst = int(round(T / dt))
    d = tgv.step(nst)
    assert np.all(d[:, 7] == 0)
    out = tgv.get()
    ue, ve, _, _ = inputs.tg2d_exact(x, y, z, T, nu)
    return max(np.abs(out[0] - ue).max(), np.abs(out[1] - ve).max())


def test_tgv_stepper_third_order_on_exact_2d_taylor_green():
    nu, T = 0.2, 1.0
    e = [_tg_error(nu, dt, T) for dt in (0.1, 0.05, 0.025)]
    rates = [math.log2(e[0] / e[1]), math.log2(e[1] / e[2])]
    assert rates[0] > 2.6 and rates[1] > 2.6, (e, rates)


def test_tgv_energy_balance():
    """dKE/dt = -2 nu Omega for periodic incompressible flow."""
    N, nel, nu, dt = 7, (4, 4, 4), 1.0 / 1600, 1e-3
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3)
    m = oracle.Mesh(N, nel, v)
    x, y, z = m.xyz
    u, vv, w, p = inputs.tgv_initial(x, y, z)
    ke0, en0 = m.diag(u, vv, w, (2 * math.pi) ** 3)
    tgv = oracle.TGV(N, nel, v, (2 * math.pi,) * 3, nu, dt, tol_v=1e-12, tol_p=1e-12,
                     abs_tol=False)
    tgv.set(u, vv, w, p)
    d = tgv.step(10)
    assert np.all(d[:, 7] == 0)
    t = d[:, 0]
    slope = (d[-1, 1] - ke0) / t[-1]
    assert abs(slope - (-2 * nu * en0)) < 0.02 * 2 * nu * en0, (slope, -2 * nu * en0)


def test_tgv_fp32_storage_mode():
    """rp = fp32 (Table 2 group B): every stored value is an FP32 number; the
    KE history moves by about the FP32 rounding of the state, no more."""
    N, nel, nu, dt = 5, (3, 3, 3), 1.0 / 1600, 1e-3
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3)
    m = oracle.Mesh(N, nel, v)
    x, y, z = m.xyz
    runs = []
    for store32 in (False, True):
        tgv = oracle.TGV(N, nel, v, (2 * math.pi,) * 3, nu, dt, tol_v=1e-12, tol_p=1e-12,
                         abs_tol=False)
        tgv.set_storage(store32)
        tgv.set(*inputs.tgv_initial(x, y, z))
        d = tgv.step(4)
        assert np.all(d[:, 7] == 0)
        runs.append((d, tgv.get()))
    (d64, s64), (d32, s32) = runs
    assert np.array_equal(s32, s32.astype(np.float32).astype(np.float64))
    assert not np.array_equal(s64, s64.astype(np.float32).astype(np.float64))
    rel = np.abs(d32[:, 1] - d64[:, 1]).max() / np.abs(d64[:, 1]).max()
    assert 0.0 < rel < 1e-6, rel


def test_variable_bdf_ext_equal_steps_are_the_textbook_coefficients():
    """Equal steps: BDF3 (11/6; 3, -3/2, 1/3) and EXT3 (3, -3, 1); BDF2 (3/2; 2, -1/2)."""
    b0, b, a = oracle.bdf_ext(3, (0.01, 0.01, 0.01))
    assert abs(b0 - 11 / 6) < 1e-14
    np.testing.assert_allclose(b, [3.0, -1.5, 1 / 3], atol=1e-13)
    np.testing.assert_allclose(a, [3.0, -3.0, 1.0], atol=1e-13)
    b0, b, a = oracle.bdf_ext(2, (0.3, 0.3))
    assert abs(b0 - 1.5) < 1e-14
    np.testing.assert_allclose(b, [2.0, -0.5, 0.0], atol=1e-14)
    np.testing.assert_allclose(a, [2.0, -1.0, 0.0], atol=1e-14)
    b0, b, a = oracle.bdf_ext(1, (0.7,))
    assert (b0, b[0], a[0]) == (1.0, 1.0, 1.0)


def test_variable_bdf2_closed_form():
    """Variable-step BDF2: b0 = (1 + 2w)/(1 + w), b1 = (1 + w), b2 = -w^2/(1 + w) with
    w = dt_{n+1}/dt_n (the textbook variable-step two-step BDF)."""
    for h0, h1 in ((0.5, 1.0), (1.0, 0.5), (0.013, 0.011)):
        w = h0 / h1
        b0, b, a = oracle.bdf_ext(2, (h0, h1))
        assert abs(b0 - (1 + 2 * w) / (1 + w)) < 1e-13
        assert abs(b[0] - (1 + w)) < 1e-13
        assert abs(b[1] + w * w / (1 + w)) < 1e-13
        np.testing.assert_allclose(a[:2], [1 + w, -w], atol=1e-13)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_variable_bdf_ext_polynomial_exactness(q):
    """On unequal steps, BDF_q differentiates degree-q polynomials exactly at
    t_{n+1} and EXT_q extrapolates degree-(q-1) polynomials exactly; one degree
    more is not exact (the order is q, not more)."""
    rng = np.random.default_rng(40 + q)
    for _ in range(5):
        dts = rng.uniform(0.2, 1.0, 3)
        t = np.array([0.0, -dts[0], -dts[0] - dts[1], -dts[:3].sum()])
        b0, b, a = oracle.bdf_ext(q, dts[:q])
        for deg in range(q + 2):
            c = rng.standard_normal(deg + 1)
            f = np.polyval(c, t)
            df = np.polyval(np.polyder(c), 0.0) if deg else 0.0
            bdf = (b0 * f[0] - sum(b[j] * f[j + 1] for j in range(q))) / dts[0]
            ext = sum(a[j] * f[j + 1] for j in range(q))
            scale = np.abs(c).sum()
            if deg <= q:
                assert abs(bdf - df) < 1e-10 * scale / dts[0], (deg, bdf, df)
            else:
                assert abs(bdf - df) > 1e-6 * scale
            if deg <= q - 1:
                assert abs(ext - f[0]) < 1e-11 * scale
            elif deg == q:
                assert abs(ext - f[0]) > 1e-6 * scale


def test_cfl_closed_forms_on_a_box():
    """A uniform velocity on an undeformed box: the CFL number is
    dt * sum_a |U_a| (2/h_a) / g, with h_a the element width and g the smallest
    GLL gap (2 at N=1, so dt * sum |U_a|/h_a, the linear-element CFL; 1 at N=2)."""
    L = (2.0, 3.0, 5.0)
    nel = (4, 3, 2)
    U = (0.7, -1.3, 0.2)
    h = [L[a] / nel[a] for a in range(3)]
    for N, g in ((1, 2.0), (2, 1.0)):
        m = mesh(N, nel, 0.0, L=L)
        uu = [np.full(m.nL, U[a]) for a in range(3)]
        c = oracle.cfl(N, m.E, m.jinv, *uu, 0.01)
        ref = 0.01 * sum(abs(U[a]) * 2 / h[a] for a in range(3)) / g
        assert abs(c - ref) < 1e-13 * ref, (N, c, ref)
    # N = 4: the smallest GLL gap is 1 - sqrt(3/7)
    m = mesh(4, nel, 0.0, L=L)
    c = oracle.cfl(4, m.E, m.jinv, *[np.full(m.nL, U[a]) for a in range(3)], 1.0)
    ref = sum(abs(U[a]) * 2 / h[a] for a in range(3)) / (1 - math.sqrt(3 / 7))
    assert abs(c - ref) < 1e-12 * ref


def test_cfl_direction_and_location():
    """Only the node's own velocity counts, and each direction is weighed by the
    gap at the node's index along it: a velocity at one interior node of N=4
    (index 2, gaps sqrt(3/7)) gives the CFL of that node alone."""
    N, nel, L = 4, (2, 2, 2), (2.0, 2.0, 2.0)
    m = mesh(N, nel, 0.0, L=L)
    n = N + 1
    u = [np.zeros(m.nL) for _ in range(3)]
    q = 3 * n ** 3 + 2 + n * 2 + n * n * 2   # element 3, node (2, 2, 2)
    u[1][q] = 2.0
    c = oracle.cfl(N, m.E, m.jinv, *u, 0.5)
    ref = 0.5 * 2.0 * (2 / 1.0) / math.sqrt(3 / 7)
    assert abs(c - ref) < 1e-13 * ref


def test_tgv_stepper_third_order_with_variable_steps():
    """Third order survives unequal steps: steps alternating 0.7h, 1.3h (plus a
    slow drift) on the exact 2-D Taylor-Green vortex converge at rate ~3."""
    nu, T, N, nel = 0.2, 1.0, 9, (4, 4, 1)
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3)
    m = oracle.Mesh(N, nel, v)
    x, y, z = m.xyz
    errs = []
    for h in (0.1, 0.05, 0.025):
        tgv = oracle.TGV(N, nel, v, (2 * math.pi,) * 3, nu, h, tol_v=1e-13, tol_p=1e-13,
                         abs_tol=False)
        for lev in (2, 1, 0):
            u, vv, w, p = inputs.tg2d_exact(x, y, z, -lev * h, nu)
            tgv.set(u, vv, w, p if lev == 0 else None, level=lev, step=2, t=0.0)
        t, k = 0.0, 0
        while T - t > 1e-12:
            dt = h * (0.7 if k % 2 == 0 else 1.3) * (1 + 0.1 * math.sin(t))
            dt = min(dt, T - t)
            tgv.set_dt(dt)
            d = tgv.step(1)
            assert d[0, 7] == 0 and abs(d[0, 8] - dt) < 1e-15
            t += dt
            k += 1
        assert abs(d[0, 0] - T) < 1e-12
        out = tgv.get()
        ue, ve, _, _ = inputs.tg2d_exact(x, y, z, T, nu)
        errs.append(max(np.abs(out[0] - ue).max(), np.abs(out[1] - ve).max()))
    rates = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert rates[0] > 2.6 and rates[1] > 2.6, (errs, rates)


def test_tgv_adaptive_step_settles_at_the_target_cfl():
    """CFL-controlled steps from a step 4x too small: the step grows by at most
    10 % a step, never past dt_max, and the CFL settles at the target."""
    N, nel, nu = 5, (3, 3, 3), 1.0 / 1600
    v = inputs.box_vertices(nel, (2 * math.pi,) * 3)
    m = oracle.Mesh(N, nel, v)
    x, y, z = m.xyz
    tgv = oracle.TGV(N, nel, v, (2 * math.pi,) * 3, nu, 0.01, tol_v=1e-10, tol_p=1e-8,
                     abs_tol=False)
    tgv.set(*inputs.tgv_initial(x, y, z))
    c0 = oracle.cfl(N, m.E, m.jinv, *inputs.tgv_initial(x, y, z)[:3], 0.01)
    tgv.set_dt(cfl_target=0.4, dt_max=1.0)
    d = tgv.step(30)
    assert np.all(d[:, 7] == 0)
    dts, cfls = d[:, 8], d[:, 9]
    assert abs(cfls[0] - c0) < 0.02 * c0          # the flow barely moves in one step
    assert np.all(dts[1:] <= 1.1 * dts[:-1] * (1 + 1e-14))
    assert np.all(dts <= 1.0)
    assert abs(cfls[-1] - 0.4) < 0.01, cfls[-5:]
    np.testing.assert_allclose(np.cumsum(dts), d[:, 0], rtol=1e-13)
