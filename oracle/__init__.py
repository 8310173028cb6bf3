"""FP64 CPU oracle for the SEM hot path (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2608_24348_gb300``); the two meet only through the seeded input
generators in ``paper_2608_24348_gb300.inputs``.

Everything is computed by ``sem_oracle.c`` and ``sem_oracle_hsmg.c`` (the
pressure solver: GMRES with the hybrid Schwarz multigrid preconditioner) --
plain C, FP64, OpenMP -- compiled on first use into
``oracle/_build/liboracle.so``.  The SEM definitions follow
the textbook spectral-element method (Deville, Fischer & Mund 2002), which is
what the paper's Neko solver implements (Sec. 2, Sec. 3); the paper prints no
SEM formula itself.  Each function's docstring names the component of the
paper it stands for.

Layouts (the oracle's own): E-vectors ``[E][N+1][N+1][N+1]`` (i fastest),
geometric factors ``G[6][nL]`` in the order (11, 22, 33, 12, 13, 23),
``jinv[9][nL]`` with ``jinv[a*3+c] = dr_a/dx_c``, coordinates ``xyz[3][nL]``.

Parity status: every function here is pinned by ``tests/test_oracle.py``
against closed forms, library routines on special cases, brute force on tiny
inputs and invariants.  The TGV stepper is pinned by the exact t=0 integrals,
the exact 2-D Taylor-Green solution and the energy balance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "sem_oracle.c"), os.path.join(_HERE, "sem_oracle_hsmg.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_BAD_MESH, ERR_NOT_CONVERGED, ERR_BREAKDOWN = 0, -1, -4, -5, -6

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_dealias_m.restype = ctypes.c_int
            L.orc_glsc3.restype = ctypes.c_double
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_cfl.restype = ctypes.c_double
            L.orc_cfl.argtypes = [ctypes.c_int, ctypes.c_long, _dp, _dp, _dp, _dp, ctypes.c_double]
            L.orc_bdf_ext_var.argtypes = [ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_double), _dp, _dp]
            L.orc_tgv_set_dt.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_set_threads.restype = None
            L.orc_glsc3.argtypes = [ctypes.c_long, ctypes.c_int, _dp, _dp, _dp]
            L.orc_ax.argtypes = [ctypes.c_int, ctypes.c_long, _dp, _dp, _dp, ctypes.c_double,
                                 ctypes.c_double, _dp, _dp]
            L.orc_pcg.argtypes = [ctypes.c_int] * 4 + [_ip, _dp, _dp, _dp, ctypes.c_double,
                                                       ctypes.c_double, _dp, _dp, ctypes.c_double,
                                                       ctypes.c_int, ctypes.c_int, _dp]
            L.orc_residual.argtypes = [ctypes.c_int] * 4 + [_ip, _dp, _dp, _dp, ctypes.c_double,
                                                            ctypes.c_double, _dp, _dp, _dp, _dp]
            L.orc_jacobi.argtypes = [ctypes.c_int] * 4 + [_ip, _dp, _dp, _dp, ctypes.c_double,
                                                          ctypes.c_double, _dp]
            L.orc_diag.argtypes = [ctypes.c_int, ctypes.c_long, _dp, _dp, _dp, ctypes.c_double,
                                   _dp, _dp, _dp, _dp]
            L.orc_tgv_create.restype = ctypes.c_void_p
            L.orc_tgv_create.argtypes = [ctypes.c_int] * 4 + [_dp, _dp, ctypes.c_double,
                                                              ctypes.c_double, ctypes.c_double,
                                                              ctypes.c_double, ctypes.c_int,
                                                              ctypes.c_int]
            L.orc_tgv_destroy.argtypes = [ctypes.c_void_p]
            L.orc_tgv_set.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp, _dp,
                                      ctypes.c_int, ctypes.c_double]
            L.orc_tgv_get.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_tgv_step.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
            L.orc_tgv_set_storage.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_fdm_1d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     _dp, _dp, _dp, _dp]
            L.orc_fdm_apply.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                                        ctypes.c_double, _dp, _dp]
            L.orc_hsmg_create.restype = ctypes.c_void_p
            L.orc_hsmg_create.argtypes = [ctypes.c_int, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _ip, _dp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int]
            L.orc_hsmg_destroy.argtypes = [ctypes.c_void_p]
            for f in ("orc_hsmg_prolong", "orc_hsmg_restrict", "orc_hsmg_smooth"):
                getattr(L, f).argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp]
            L.orc_hsmg_apply.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_hsmg_coarse_stats.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_hsmg_coarse_stats.restype = None
            L.orc_fgmres.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4 + [_ip, _dp, _dp, _dp,
                                                                              ctypes.c_double,
                                                                              ctypes.c_double, _dp, _dp,
                                                                              ctypes.c_double,
                                                                              ctypes.c_int, ctypes.c_int,
                                                                              ctypes.c_int, _dp, _dp]
            _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle wants C-contiguous f64"
    return a.ctypes.data_as(_dp)


def _ipt(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# 1-D tools
# ----------------------------------------------------------------------------

def gll(N: int):
    """GLL nodes and weights on [-1, 1] (the SEM basis of Neko, Sec. 2)."""
    xi = np.zeros(N + 1); w = np.zeros(N + 1)
    rc = lib().orc_gll(N, _p(xi), _p(w))
    if rc:
        raise ValueError(f"orc_gll({N}) -> {rc}")
    return xi, w


def gl(M: int):
    """Gauss-Legendre points and weights (dealiasing grid of adv_dealias)."""
    eta = np.zeros(M); w = np.zeros(M)
    rc = lib().orc_gl(M, _p(eta), _p(w))
    if rc:
        raise ValueError(f"orc_gl({M}) -> {rc}")
    return eta, w


def deriv(N: int) -> np.ndarray:
    """GLL derivative matrix D[i, j] = l_j'(xi_i)."""
    xi, _ = gll(N)
    D = np.zeros((N + 1, N + 1))
    lib().orc_deriv(N, _p(xi), _p(D))
    return D


def interp(N: int, x) -> np.ndarray:
    """Lagrange interpolation matrix J[q, j] = l_j(x_q) on the GLL nodes."""
    xi, _ = gll(N)
    x = _f64(x)
    J = np.zeros((len(x), N + 1))
    lib().orc_interp(N, _p(xi), len(x), _p(x), _p(J))
    return J


def fourier(K, cc, cs, x, y, z):
    """sum_m cc_m cos(k_m . x) + cs_m sin(k_m . x) at the given points."""
    K = np.ascontiguousarray(K, dtype=np.int64)
    cc, cs = _f64(cc), _f64(cs)
    x, y, z = (_f64(v).reshape(-1) for v in (x, y, z))
    out = np.zeros(x.size)
    kmax = int(np.abs(K).max())
    rc = lib().orc_fourier(ctypes.c_long(len(K)), K.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                           _p(cc), _p(cs), ctypes.c_long(x.size), _p(x), _p(y), _p(z), kmax, _p(out))
    if rc:
        raise ValueError(f"orc_fourier -> {rc}")
    return out


def bdf_ext(q, dts):
    """Variable-step (b0, b[3], a[3]) of order q for the steps dts = (dt_{n+1}, dt_n, dt_{n-1})."""
    dts = _f64(list(dts) + [1.0] * (3 - len(dts)))
    b0 = ctypes.c_double()
    b, a = np.zeros(3), np.zeros(3)
    lib().orc_bdf_ext_var(int(q), _p(dts), ctypes.byref(b0), _p(b), _p(a))
    return b0.value, b, a


def cfl(N, E, jinv, u, v, w, dt):
    """CFL number of (u, v, w) for step dt (reference-space speed over the GLL spacing)."""
    return lib().orc_cfl(int(N), int(E), _p(_f64(jinv)), _p(_f64(u)), _p(_f64(v)), _p(_f64(w)), float(dt))


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return lib().orc_threads()


def set_threads(n: int) -> None:
    """OpenMP threads of later oracle calls (for timing the baseline)."""
    lib().orc_set_threads(int(n))


def dealias_m(N: int) -> int:
    """Points per direction of the 3/2-rule dealiasing grid."""
    return lib().orc_dealias_m(N)


# ----------------------------------------------------------------------------
# Mesh, geometry, operator, gather-scatter
# ----------------------------------------------------------------------------

class Mesh:
    """A structured nelx x nely x nelz hexahedral mesh with its FP64 geometry.

    ``vert`` is the vertex grid ``[(nelz+1), (nely+1), (nelx+1), 3]``.
    """

    def __init__(self, N, nel, vert, periodic=(1, 1, 1)):
        self.N = int(N)
        self.nel = tuple(int(v) for v in nel)
        self.periodic = tuple(int(bool(p)) for p in periodic)
        self.n = self.N + 1
        self.n3 = self.n ** 3
        self.E = self.nel[0] * self.nel[1] * self.nel[2]
        self.nL = self.E * self.n3
        self.vert = _f64(vert).reshape(-1)
        assert self.vert.size == (self.nel[0] + 1) * (self.nel[1] + 1) * (self.nel[2] + 1) * 3
        self.D = deriv(self.N)
        self.xyz = np.zeros((3, self.nL))
        self.jinv = np.zeros((9, self.nL))
        self.G = np.zeros((6, self.nL))
        self.B = np.zeros(self.nL)
        rc = lib().orc_geom(self.N, *self.nel, _p(self.vert), _p(self.xyz), _p(self.jinv),
                            _p(self.G), _p(self.B))
        if rc == ERR_BAD_MESH:
            raise ValueError("non-positive Jacobian determinant")
        if rc:
            raise ValueError(f"orc_geom -> {rc}")
        self.mult = self.dssum(np.ones(self.nL))
        self.imult = 1.0 / self.mult

    # local operator (ax_helm)
    def ax(self, u, h1=1.0, h2=0.0):
        u = _f64(u).reshape(-1)
        w = np.zeros(self.nL)
        lib().orc_ax(self.N, self.E, _p(self.D), _p(self.G), _p(self.B), h1, h2, _p(u), _p(w))
        return w

    def dssum(self, u):
        """Direct-stiffness sum Q Q^T u (returns a new array)."""
        out = _f64(u).reshape(-1).copy()
        per, pp = _ipt(self.periodic)
        lib().orc_dssum(self.N, *self.nel, pp, _p(out))
        return out

    def glsc3(self, a, b, c=None):
        """sum a b c; with c = None the weights are 1/mult (assembled product)."""
        c = self.imult if c is None else _f64(c)
        return lib().orc_glsc3(self.E, self.n3, _p(_f64(a)), _p(_f64(b)), _p(c))

    def jacobi(self, h1=1.0, h2=0.0):
        """1 / dssum(diag(A)) including the face cross terms."""
        out = np.zeros(self.nL)
        per, pp = _ipt(self.periodic)
        lib().orc_jacobi(self.N, *self.nel, pp, _p(self.D), _p(self.G), _p(self.B), h1, h2,
                         _p(out))
        return out

    def pcg(self, b, h1=1.0, h2=0.0, x0=None, tol=1e-10, abs_tol=False, maxit=20000):
        """Jacobi-PCG on dssum(A) x = b; returns (x, info dict)."""
        b = _f64(b).reshape(-1)
        x = np.zeros(self.nL) if x0 is None else _f64(x0).reshape(-1).copy()
        out = np.zeros(3)
        per, pp = _ipt(self.periodic)
        rc = lib().orc_pcg(self.N, *self.nel, pp, _p(self.D), _p(self.G), _p(self.B), h1, h2,
                           _p(b), _p(x), tol, int(abs_tol), maxit, _p(out))
        return x, {"status": rc, "iters": int(out[0]), "rnorm": out[1], "bnorm": out[2]}

    def residual(self, b, x, h1=1.0, h2=0.0):
        """(||b' - dssum(A x)||, ||b'||), b' = b minus its mean when h2 == 0."""
        out = np.zeros(2)
        per, pp = _ipt(self.periodic)
        lib().orc_residual(self.N, *self.nel, pp, _p(self.D), _p(self.G), _p(self.B), h1, h2,
                           _p(_f64(b).reshape(-1)), _p(_f64(x).reshape(-1)), None, _p(out))
        return out[0], out[1]

    def convect(self, u, v, w):
        """Weak 3/2-rule dealiased (u . grad) u_c, local (not assembled)."""
        C = np.zeros((3, self.nL))
        lib().orc_convect(self.N, *self.nel, _p(self.vert), _p(self.jinv),
                          _p(_f64(u).reshape(-1)), _p(_f64(v).reshape(-1)),
                          _p(_f64(w).reshape(-1)), _p(C[0]), _p(C[1]), _p(C[2]))
        return C

    def diag(self, u, v, w, V):
        """(kinetic energy, enstrophy), both 1/(2V) sum_local B |.|^2."""
        out = np.zeros(2)
        lib().orc_diag(self.N, self.E, _p(self.D), _p(self.jinv), _p(self.B), V,
                       _p(_f64(u).reshape(-1)), _p(_f64(v).reshape(-1)),
                       _p(_f64(w).reshape(-1)), _p(out))
        return out[0], out[1]


# ----------------------------------------------------------------------------
# TGV stepper
# ----------------------------------------------------------------------------

class TGV:
    """BDF3/EXT3 P_N-P_N stepper with 3/2 dealiasing on a periodic box."""

    def __init__(self, N, nel, vert, L, nu, dt, tol_v=1e-6, tol_p=1e-4, abs_tol=True,
                 maxit=20000):
        self.N, self.nel = int(N), tuple(int(v) for v in nel)
        self.nL = self.nel[0] * self.nel[1] * self.nel[2] * (self.N + 1) ** 3
        self._vert = _f64(vert).reshape(-1)
        L = _f64(L)
        h = lib().orc_tgv_create(self.N, *self.nel, _p(self._vert), _p(L), nu, dt, tol_v, tol_p,
                                 int(abs_tol), maxit)
        if not h:
            raise ValueError("orc_tgv_create failed")
        self._h = ctypes.c_void_p(h)

    def set(self, u, v, w, p=None, level=0, step=0, t=0.0):
        """Set u^{n-level} (and p^n, the step count and the time for level 0)."""
        pp = _p(_f64(p).reshape(-1)) if p is not None else None
        lib().orc_tgv_set(self._h, level, _p(_f64(u).reshape(-1)), _p(_f64(v).reshape(-1)),
                          _p(_f64(w).reshape(-1)), pp, step, t)

    def get(self):
        out = np.zeros((4, self.nL))
        lib().orc_tgv_get(self._h, _p(out[0]), _p(out[1]), _p(out[2]), _p(out[3]))
        return out

    def set_storage(self, store32):
        """store32: keep the stored state as FP32 values (rp = fp32, Table 2 group B)."""
        lib().orc_tgv_set_storage(self._h, int(bool(store32)))

    def set_dt(self, dt=0.0, cfl_target=0.0, dt_max=0.0):
        """Step of the next step (dt > 0) and the adaptive rule (cfl_target > 0)."""
        lib().orc_tgv_set_dt(self._h, float(dt), float(cfl_target), float(dt_max))

    def step(self, nsteps=1):
        """Advance; returns diag rows {t, KE, enstrophy, it_p, it_u, it_v, it_w, status, dt, CFL}."""
        d = np.zeros((nsteps, 10))
        lib().orc_tgv_step(self._h, nsteps, _p(d))
        return d

    def __del__(self):
        try:
            lib().orc_tgv_destroy(self._h)
        except Exception:
            pass


# ----------------------------------------------------------------------------
# Pressure solver: flexible GMRES with the hybrid Schwarz multigrid (Sec. 1, Sec. 3)
# ----------------------------------------------------------------------------

def fdm_1d(N, h, hl=0.0, hr=0.0):
    """1-D factors of the fast-diagonalisation local solve: (S, lam, K, Mdiag) with
    K S = M S diag(lam), S^T M S = I (K, M: the element's 1-D stiffness and mass,
    extended to the neighbours' first interior GLL nodes; hl, hr = 0: no neighbour)."""
    n = N + 1
    S, lam, K, M = np.zeros((n, n)), np.zeros(n), np.zeros((n, n)), np.zeros(n)
    rc = lib().orc_fdm_1d(int(N), float(h), float(hl), float(hr), _p(S), _p(lam), _p(K), _p(M))
    if rc != OK:
        raise ValueError(f"orc_fdm_1d: {rc}")
    return S, lam, K, M


def fdm_apply(N, factors, h1, h2, r):
    """A~^{-1} r on one element from three directions' (S, lam) factors."""
    (Sx, lx), (Sy, ly), (Sz, lz) = [(_f64(S), _f64(lam)) for S, lam in factors]
    z = np.zeros((N + 1) ** 3)
    lib().orc_fdm_apply(int(N), _p(Sx), _p(lx), _p(Sy), _p(ly), _p(Sz), _p(lz), float(h1),
                        float(h2), _p(_f64(r).reshape(-1)), _p(z))
    return z


class HSMG:
    """Hybrid Schwarz multigrid hierarchy of orders `orders` (finest first) on a mesh."""

    def __init__(self, orders, nel, vert, periodic=(1, 1, 1), h1=1.0, h2=0.0, ctol=1e-2,
                 cmaxit=1000):
        self.orders = [int(o) for o in orders]
        self.nel = tuple(int(v) for v in nel)
        self.E = self.nel[0] * self.nel[1] * self.nel[2]
        self._o, op = _ipt(self.orders)
        self._pd, pp = _ipt([int(bool(p)) for p in periodic])
        self._vert = _f64(vert).reshape(-1)
        h = lib().orc_hsmg_create(len(self.orders), op, *self.nel, pp, _p(self._vert), float(h1),
                                  float(h2), float(ctol), int(cmaxit))
        if not h:
            raise ValueError("orc_hsmg_create rejected the hierarchy")
        self._h = ctypes.c_void_p(h)

    def nL(self, level=0):
        return self.E * (self.orders[level] + 1) ** 3

    def apply(self, r):
        z = np.zeros(self.nL())
        lib().orc_hsmg_apply(self._h, _p(_f64(r).reshape(-1)), _p(z))
        return z

    def smooth(self, level, r):
        z = np.zeros(self.nL(level))
        lib().orc_hsmg_smooth(self._h, int(level), _p(_f64(r).reshape(-1)), _p(z))
        return z

    def prolong(self, level, u):
        out = np.zeros(self.nL(level))
        lib().orc_hsmg_prolong(self._h, int(level), _p(_f64(u).reshape(-1)), _p(out))
        return out

    def restrict(self, level, r):
        out = np.zeros(self.nL(level + 1))
        lib().orc_hsmg_restrict(self._h, int(level), _p(_f64(r).reshape(-1)), _p(out))
        return out

    def coarse_stats(self):
        a, b = np.zeros(1), np.zeros(1)
        lib().orc_hsmg_coarse_stats(self._h, _p(a), _p(b))
        return int(a[0]), int(b[0])

    def __del__(self):
        try:
            lib().orc_hsmg_destroy(self._h)
        except Exception:
            pass


def fgmres(b, x0=None, hsmg=None, mesh=None, h1=1.0, h2=0.0, tol=1e-10, abs_tol=False, m=30,
           maxit=1000, history=False):
    """Flexible GMRES(m) on the finest level of `hsmg` (preconditioned by it) or on
    `mesh` (an oracle Mesh, no preconditioner).  Returns (x, status, info) with info
    = {iters, rnorm, bnorm, restarts} (and "hist", the Arnoldi residual estimates)."""
    b = _f64(b).reshape(-1)
    x = np.zeros_like(b) if x0 is None else _f64(x0).reshape(-1).copy()
    out = np.zeros(4)
    hist = np.zeros(maxit + 1) if history else None
    if hsmg is not None:
        pd, pp = _ipt([1, 1, 1])
        st = lib().orc_fgmres(hsmg._h, 0, 0, 0, 0, pp, None, None, None, 0.0, 0.0, _p(b), _p(x),
                              float(tol), int(bool(abs_tol)), int(m), int(maxit), _p(out),
                              _p(hist) if history else None)
    else:
        pd, pp = _ipt(mesh.periodic)
        st = lib().orc_fgmres(None, mesh.N, *mesh.nel, pp, _p(mesh.D), _p(mesh.G), _p(mesh.B),
                              float(h1), float(h2), _p(b), _p(x), float(tol), int(bool(abs_tol)),
                              int(m), int(maxit), _p(out), _p(hist) if history else None)
    info = dict(iters=int(out[0]), rnorm=float(out[1]), bnorm=float(out[2]), restarts=int(out[3]))
    if history:
        info["hist"] = hist[:info["iters"] + 1]
    return x, st, info
