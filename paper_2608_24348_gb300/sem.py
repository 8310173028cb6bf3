"""Thin ctypes binding of libsem (``include/sem.h``): argument marshalling only.

Every computation runs in the CUDA library; this module converts tensors and
arrays to pointers and error codes to exceptions.  Field arguments may be
torch CUDA tensors (device pointers, the fast path), or torch CPU tensors /
numpy arrays (host pointers, staged by the library).  ``load()`` raises if the
library cannot be built or loaded: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

F64, F32, BF16_TC, F16_TC, F64_NATIVE, F16X2_TC, BF16X3_TC, F32_TUNED = 0, 1, 2, 3, 4, 5, 6, 7
DTYPES = {"f64": F64, "f32": F32, "bf16_tc": BF16_TC, "f16_tc": F16_TC, "f64_native": F64_NATIVE,
          "f16x2_tc": F16X2_TC, "bf16x3_tc": BF16X3_TC, "f32_tuned": F32_TUNED}

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_BAD_MESH, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
ERR_TOO_LARGE = -8
NOALLOC_MAX_NODES = 1000000
TUNE_MAX = 16  # entries of sem_tune_ax's ms array (SEM_TUNE_MAX)

_lib = None
_lock = threading.Lock()


class SemError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = _lib.sem_strerror(code).decode() if _lib else str(code)
        detail = _lib.sem_last_cuda_error().decode() if (_lib and code == ERR_CUDA) else ""
        super().__init__(f"{where}: {msg} ({code}) {detail}".strip())


class CtxInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("nelx", ctypes.c_int), ("nely", ctypes.c_int),
                ("nelz", ctypes.c_int), ("periodic", ctypes.c_int * 3), ("E", ctypes.c_int64),
                ("nL", ctypes.c_int64), ("nG", ctypes.c_int64), ("volume", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("abs_tol", ctypes.c_int), ("maxit", ctypes.c_int),
                ("inner", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("wait_timeout_s", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("final_rnorm", ctypes.c_double), ("bnorm", ctypes.c_double)]

    def as_dict(self):
        return {"status": self.status, "iters": self.iters, "outer_iters": self.outer_iters,
                "rnorm": self.final_rnorm, "bnorm": self.bnorm}


class TgvPolicy(ctypes.Structure):
    _fields_ = [("first_step", ctypes.c_int), ("sem", ctypes.c_int), ("vel", ctypes.c_int),
                ("pres", ctypes.c_int), ("storage", ctypes.c_int)]


class TgvDiag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("ke", ctypes.c_double), ("enstrophy", ctypes.c_double),
                ("iters", ctypes.c_int * 4), ("status", ctypes.c_int), ("dt", ctypes.c_double),
                ("cfl", ctypes.c_double)]


EXPORTS = ["sem_setup", "sem_destroy", "sem_get_info", "sem_strerror", "sem_coords", "sem_geom",
           "sem_ax", "sem_dssum", "sem_jacobi", "sem_solve_opts_default", "sem_pcg_solve",
           "sem_last_solve_info", "sem_pcg_solve_batched", "sem_tgv_init", "sem_tgv_set",
           "sem_tgv_step", "sem_tgv_get", "sem_tgv_energy", "sem_tgv_destroy",
           "sem_pcg_solve_noalloc", "sem_device_status", "sem_tune_ax", "sem_set_ax_variant",
           "sem_tgv_set_policy", "sem_tgv_set_projection", "sem_tune_inner", "sem_set_inner_path",
           "sem_tgv_set_dt", "sem_hsmg_create", "sem_hsmg_apply", "sem_gmres_solve",
           "sem_hsmg_destroy", "sem_tgv_set_pressure_solver"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsem.so (building it with nvcc if needed); raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsem.so not found at {path}; the CUDA extension is required")
        L = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        L.sem_strerror.restype = ctypes.c_char_p
        L.sem_strerror.argtypes = [ctypes.c_int]
        L.sem_last_cuda_error.restype = ctypes.c_char_p
        L.sem_setup.argtypes = [ctypes.c_int] * 4 + [dp, ip, dp, ctypes.POINTER(vp)]
        L.sem_destroy.argtypes = [vp]
        L.sem_destroy.restype = None
        L.sem_get_info.argtypes = [vp, ctypes.POINTER(CtxInfo)]
        L.sem_device_status.argtypes = [vp]
        L.sem_tune_ax.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, ip]
        L.sem_set_ax_variant.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.sem_tune_inner.argtypes = [vp, ctypes.c_int, dp, ip]
        L.sem_set_inner_path.argtypes = [ctypes.c_int, ctypes.c_int]
        L.sem_coords.argtypes = [vp, vp, vp]
        L.sem_geom.argtypes = [vp, vp, vp]
        L.sem_ax.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
        L.sem_dssum.argtypes = [vp, vp, ctypes.c_int, vp]
        L.sem_jacobi.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp]
        L.sem_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
        L.sem_solve_opts_default.restype = None
        L.sem_pcg_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
        L.sem_last_solve_info.argtypes = [vp, ctypes.POINTER(SolveInfo)]
        L.sem_pcg_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(vp), dp, dp, ctypes.POINTER(SolveOpts),
                                            ctypes.POINTER(SolveInfo), vp]
        L.sem_tgv_init.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveOpts),
                                   ctypes.POINTER(vp)]
        L.sem_tgv_set.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
        L.sem_tgv_step.argtypes = [vp, ctypes.c_int, ctypes.POINTER(TgvDiag), vp]
        L.sem_tgv_get.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sem_tgv_energy.argtypes = [vp, dp, dp, vp]
        L.sem_tgv_destroy.argtypes = [vp]
        L.sem_tgv_set_policy.argtypes = [vp, ctypes.c_int, ctypes.POINTER(TgvPolicy)]
        L.sem_tgv_set_projection.argtypes = [vp, ctypes.c_int]
        L.sem_tgv_set_dt.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.sem_hsmg_create.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(vp)]
        L.sem_hsmg_apply.argtypes = [vp, vp, vp, vp]
        L.sem_gmres_solve.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(SolveOpts), ctypes.c_int,
                                      ctypes.POINTER(SolveInfo), vp]
        L.sem_hsmg_destroy.argtypes = [vp]
        L.sem_hsmg_destroy.restype = None
        L.sem_tgv_set_pressure_solver.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.sem_tgv_destroy.restype = None
        L.sem_pcg_solve_noalloc.argtypes = [ctypes.c_int] * 4 + [ip, vp, vp, vp, ctypes.c_double,
                                                                 ctypes.c_double,
                                                                 ctypes.POINTER(SolveOpts),
                                                                 ctypes.POINTER(SolveInfo), vp]
        _lib = L
        return L


def _check(rc, where):
    if rc != OK:
        raise SemError(rc, where)


def ptr(x):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "fields must be contiguous"
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        assert x.flags["C_CONTIGUOUS"], "fields must be contiguous"
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_ptr(stream=None):
    """cudaStream_t of a torch stream (default: torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def opts(tol=1e-10, abs_tol=False, maxit=20000, inner="f64", inner_tol=1e-4, max_outer=50,
         wait_timeout_s=0.0):
    o = SolveOpts()
    o.tol, o.abs_tol, o.maxit = tol, int(abs_tol), maxit
    o.inner = DTYPES[inner] if isinstance(inner, str) else int(inner)
    o.inner_tol, o.max_outer, o.wait_timeout_s = inner_tol, max_outer, wait_timeout_s
    return o


class Ctx:
    """A libsem context (geometry + workspaces on the current CUDA device)."""

    def __init__(self, N, nel, extents=(6.283185307179586,) * 3, periodic=(1, 1, 1),
                 vertices=None):
        L = load()
        import numpy as np
        ext = (ctypes.c_double * 3)(*[float(v) for v in extents])
        per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
        self._vert = None
        vp = None
        if vertices is not None:
            self._vert = np.ascontiguousarray(vertices, dtype=np.float64)
            vp = self._vert.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(L.sem_setup(int(N), int(nel[0]), int(nel[1]), int(nel[2]), ext, per, vp,
                           ctypes.byref(h)), "sem_setup")
        self._h = h
        inf = CtxInfo()
        _check(L.sem_get_info(h, ctypes.byref(inf)), "sem_get_info")
        self.N, self.nel = inf.N, (inf.nelx, inf.nely, inf.nelz)
        self.E, self.nL, self.nG, self.volume = inf.E, inf.nL, inf.nG, inf.volume
        self.periodic = tuple(inf.periodic)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.sem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self):
        """SEM_OK, or SEM_ERR_TIMEOUT if a bounded wait of a staged kernel gave up."""
        return _lib.sem_device_status(self._h)

    # -- setup exports
    def coords(self, out, stream=None):
        _check(_lib.sem_coords(self._h, ptr(out), _sp(out, stream)), "sem_coords")
        return out

    def geom(self, out, stream=None):
        _check(_lib.sem_geom(self._h, ptr(out), _sp(out, stream)), "sem_geom")
        return out

    # -- operators
    def ax(self, u, w, h1=1.0, h2=0.0, dtype="f64", stream=None):
        dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        _check(_lib.sem_ax(self._h, ptr(u), ptr(w), float(h1), float(h2), dt, _sp(u, stream)),
               "sem_ax")
        return w

    def dssum(self, u, dtype="f64", stream=None):
        dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        _check(_lib.sem_dssum(self._h, ptr(u), dt, _sp(u, stream)), "sem_dssum")
        return u

    def jacobi(self, out, h1=1.0, h2=0.0, stream=None):
        _check(_lib.sem_jacobi(self._h, float(h1), float(h2), ptr(out), _sp(out, stream)),
               "sem_jacobi")
        return out

    # -- solvers
    def pcg_solve(self, b, x, h1=1.0, h2=0.0, sync=True, stream=None, **kw):
        o = opts(**kw)
        info = SolveInfo()
        rc = _lib.sem_pcg_solve(self._h, ptr(b), ptr(x), float(h1), float(h2), ctypes.byref(o),
                                ctypes.byref(info) if sync else None, _sp(b, stream))
        if not sync:
            _check(rc, "sem_pcg_solve")
            return None
        if rc not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT):
            _check(rc, "sem_pcg_solve")
        return info.as_dict()

    def last_solve_info(self):
        info = SolveInfo()
        _check(_lib.sem_last_solve_info(self._h, ctypes.byref(info)), "sem_last_solve_info")
        return info.as_dict()


class HSMG:
    """Hybrid Schwarz multigrid preconditioner and flexible GMRES on a context."""

    def __init__(self, ctx, orders, h1=1.0, h2=0.0, dtype="f32", coarse_tol=0.1, coarse_maxit=200):
        self.ctx = ctx
        o = (ctypes.c_int * len(orders))(*[int(v) for v in orders])
        h = ctypes.c_void_p()
        _check(_lib.sem_hsmg_create(ctx.handle, len(orders), o, float(h1), float(h2), DTYPES[dtype],
                                    float(coarse_tol), int(coarse_maxit), ctypes.byref(h)),
               "sem_hsmg_create")
        self._h = h

    def apply(self, r, z, stream=None):
        _check(_lib.sem_hsmg_apply(self._h, ptr(r), ptr(z), _sp(r, stream)), "sem_hsmg_apply")

    def gmres(self, b, x, restart=30, precond=True, stream=None, **kw):
        o = opts(**kw)
        info = SolveInfo()
        rc = _lib.sem_gmres_solve(self._h, int(bool(precond)), ptr(b), ptr(x), ctypes.byref(o),
                                  int(restart), ctypes.byref(info), _sp(b, stream))
        if rc not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(rc, "sem_gmres_solve")
        return info.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.sem_hsmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _sp(t, stream):
    """Stream handle for a call: torch's current stream for CUDA tensors, else NULL."""
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    if hasattr(t, "is_cuda") and t.is_cuda:
        return stream_ptr()
    return None


def pcg_solve_batched(ctxs, bs, xs, h1s, h2s, sync=True, stream=None, **kw):
    n = len(ctxs)
    o = opts(**kw)
    arr_c = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    arr_b = (ctypes.c_void_p * n)(*[ptr(b) for b in bs])
    arr_x = (ctypes.c_void_p * n)(*[ptr(x) for x in xs])
    h1 = (ctypes.c_double * n)(*[float(v) for v in h1s])
    h2 = (ctypes.c_double * n)(*[float(v) for v in h2s])
    infos = (SolveInfo * n)()
    rc = _lib.sem_pcg_solve_batched(n, arr_c, arr_b, arr_x, h1, h2, ctypes.byref(o),
                                    infos if sync else None, _sp(bs[0], stream))
    if not sync:
        _check(rc, "sem_pcg_solve_batched")
        return None
    if rc not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT):
        _check(rc, "sem_pcg_solve_batched")
    return [infos[i].as_dict() for i in range(n)]


def pcg_solve_noalloc(N, nel, periodic, geom, b, x, h1=1.0, h2=0.0, stream=None, **kw):
    """FP64 PCG without any allocation (scratch in a fixed static device array).

    geom: device FP64 tensor [E][7][(N+1)^3]; b, x: device FP64 E-vectors.
    Synchronous; returns the info dict (raises on argument / CUDA errors)."""
    L = load()
    o = opts(**kw)
    info = SolveInfo()
    per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
    rc = L.sem_pcg_solve_noalloc(int(N), int(nel[0]), int(nel[1]), int(nel[2]), per, ptr(geom),
                                 ptr(b), ptr(x), float(h1), float(h2), ctypes.byref(o),
                                 ctypes.byref(info), _sp(b, stream))
    if rc not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT):
        _check(rc, "sem_pcg_solve_noalloc")
    return info.as_dict()


def set_ax_variant(N, dtype, variant):
    """Select sem_ax's kernel for order N and dtype in this process (-1: the
    built-in default)."""
    L = load()
    _check(L.sem_set_ax_variant(int(N), DTYPES[dtype] if isinstance(dtype, str) else int(dtype),
                                int(variant)), "sem_set_ax_variant")


def autotune(ctx, dtype="f32", reps=5, cache=None):
    """Pick sem_ax's kernel for ctx's order and dtype by timing the candidates.

    cache: path of a JSON file keyed by (GPU name, N, dtype); a cached choice is
    applied without timing, a new one is written back.  Returns
    {"variant": v, "ms": [per candidate], "cached": bool}."""
    import json
    import torch
    L = load()
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    key = f"{torch.cuda.get_device_name()}|N={ctx.N}|dtype={dt}"
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            set_ax_variant(ctx.N, dt, table[key]["variant"])
            return dict(table[key], cached=True)
    ms = (ctypes.c_double * TUNE_MAX)(*([-1.0] * TUNE_MAX))
    best = ctypes.c_int()
    _check(L.sem_tune_ax(ctx.handle, dt, int(reps), ms, ctypes.byref(best)), "sem_tune_ax")
    out = {"variant": best.value, "ms": [ms[i] for i in range(TUNE_MAX) if ms[i] >= 0]}
    if cache:
        table[key] = out
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return dict(out, cached=False)


def set_inner_path(N, path):
    """Inner path of order N for inner="f32_tuned": 0 FP32 CUDA cores, 1 split FP16 tensor cores."""
    _check(load().sem_set_inner_path(int(N), int(path)), "sem_set_inner_path")


def tune_inner(ctx, iters=30, cache=None):
    """Pick the inner path of refinement for ctx's order by timing both candidates
    (sem_tune_inner).  cache: JSON file keyed by (GPU name, N); a cached choice
    is applied without timing.  Returns {"path": p, "ms_per_iter": [fp32, tc],
    "cached": bool}."""
    import json
    import torch
    L = load()
    key = f"{torch.cuda.get_device_name()}|N={ctx.N}|inner"
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            set_inner_path(ctx.N, table[key]["path"])
            return dict(table[key], cached=True)
    ms = (ctypes.c_double * 2)(-1.0, -1.0)
    best = ctypes.c_int()
    _check(L.sem_tune_inner(ctx.handle, int(iters), ms, ctypes.byref(best)), "sem_tune_inner")
    out = {"path": best.value, "ms_per_iter": [ms[0], ms[1]]}
    if cache:
        table[key] = out
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return dict(out, cached=False)


class TGV:
    """Taylor-Green vortex stepper bound to a periodic context."""

    def __init__(self, ctx, nu, dt, op="f64", vel=None, pres=None):
        self.ctx = ctx
        h = ctypes.c_void_p()
        vo = vel if vel is not None else opts(tol=1e-6, abs_tol=True)
        po = pres if pres is not None else opts(tol=1e-4, abs_tol=True,
                                                inner="f32" if op == "f32" else "f64")
        _check(_lib.sem_tgv_init(ctx.handle, float(nu), float(dt), DTYPES[op], ctypes.byref(vo),
                                 ctypes.byref(po), ctypes.byref(h)), "sem_tgv_init")
        self._h = h

    def set_policy(self, rules):
        """Precision schedule: a list of dicts with keys first_step (default 1),
        sem, vel, pres, storage (names of DTYPES; defaults f64); [] restores the
        precisions given at construction."""
        arr = (TgvPolicy * max(1, len(rules)))()
        for k, r in enumerate(rules):
            arr[k] = TgvPolicy(int(r.get("first_step", 1)), DTYPES[r.get("sem", "f64")],
                               DTYPES[r.get("vel", "f64")], DTYPES[r.get("pres", "f64")],
                               DTYPES[r.get("storage", "f64")])
        _check(_lib.sem_tgv_set_policy(self._h, len(rules), arr), "sem_tgv_set_policy")

    def set_projection(self, max_vectors):
        """Keep up to max_vectors earlier pressure solutions for projection (0 = off)."""
        _check(_lib.sem_tgv_set_projection(self._h, int(max_vectors)), "sem_tgv_set_projection")

    def set_dt(self, dt=0.0, cfl_target=0.0, dt_max=0.0):
        """Size of the next step (dt > 0) and the CFL-controlled step
        (cfl_target > 0: each next step from the last step's CFL number, capped
        by dt_max > 0; 0 keeps the step fixed)."""
        _check(_lib.sem_tgv_set_dt(self._h, float(dt), float(cfl_target), float(dt_max)),
               "sem_tgv_set_dt")

    def set_pressure_solver(self, kind="gmres_hsmg", restart=30, vcycle="f32"):
        """Pressure solver: "pcg" (Jacobi-PCG, the default) or "gmres_hsmg" (flexible
        GMRES with the hybrid Schwarz multigrid, V-cycle in `vcycle` precision)."""
        k = {"pcg": 0, "gmres_hsmg": 1}[kind]
        _check(_lib.sem_tgv_set_pressure_solver(self._h, k, int(restart), DTYPES[vcycle]),
               "sem_tgv_set_pressure_solver")

    def set(self, u, v, w, p=None, level=0, step=0, t=0.0, stream=None):
        _check(_lib.sem_tgv_set(self._h, level, ptr(u), ptr(v), ptr(w), ptr(p), step, t,
                                _sp(u, stream)), "sem_tgv_set")

    def step(self, nsteps=1, diag=True, stream=None):
        import torch
        sp = stream_ptr(stream) if torch.cuda.is_available() else None
        if diag:
            d = (TgvDiag * nsteps)()
            rc = _lib.sem_tgv_step(self._h, nsteps, d, sp)
            if rc not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT):
                _check(rc, "sem_tgv_step")
            return [{"t": x.t, "ke": x.ke, "enstrophy": x.enstrophy, "iters": list(x.iters),
                     "status": x.status, "dt": x.dt, "cfl": x.cfl} for x in d]
        _check(_lib.sem_tgv_step(self._h, nsteps, None, sp), "sem_tgv_step")
        return None

    def get(self, u=None, v=None, w=None, p=None, stream=None):
        t = next(x for x in (u, v, w, p) if x is not None)
        _check(_lib.sem_tgv_get(self._h, ptr(u), ptr(v), ptr(w), ptr(p), _sp(t, stream)),
               "sem_tgv_get")

    def energy(self, stream=None):
        ke, en = ctypes.c_double(), ctypes.c_double()
        _check(_lib.sem_tgv_energy(self._h, ctypes.byref(ke), ctypes.byref(en),
                                   stream_ptr(stream)), "sem_tgv_energy")
        return ke.value, en.value

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.sem_tgv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
