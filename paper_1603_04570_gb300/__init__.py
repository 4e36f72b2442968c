"""Python binding of libok_gb300.so (include/ok.h): argument marshalling only.

Every computation runs in the CUDA library.  Arrays may be torch tensors
(CUDA or CPU) or numpy arrays; they must be float64 and contiguous.  The
functions keep the C names (``ok_grid_create``, ``ok_timestep``, ...);
``Grid`` wraps a handle for convenience.

If the library cannot be built or loaded this module raises: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_char_p, c_double, c_int, c_longlong, c_void_p

from . import _build

OK_SUCCESS, OK_ERR_INVALID_ARG, OK_ERR_NOMEM, OK_ERR_CUDA = 0, 1, 2, 3
OK_ERR_NOT_CONVERGED, OK_ERR_NONFINITE, OK_ERR_TIMEOUT, OK_ERR_INTERNAL = 4, 5, 6, 7
OK_FP64, OK_MIXED, OK_MIXED_HALF = 0, 1, 2
STATUS_NAMES = {0: "OK_SUCCESS", 1: "OK_ERR_INVALID_ARG", 2: "OK_ERR_NOMEM", 3: "OK_ERR_CUDA",
                4: "OK_ERR_NOT_CONVERGED", 5: "OK_ERR_NONFINITE", 6: "OK_ERR_TIMEOUT", 7: "OK_ERR_INTERNAL"}


class Params(Structure):
    _fields_ = [("eps", c_double), ("sigma", c_double), ("m", c_double), ("theta", c_double), ("dt", c_double)]


class Opts(Structure):
    _fields_ = [("restart", c_int), ("max_gmres", c_int), ("max_newton", c_int), ("newton_extra", c_int),
                ("q_A", c_int), ("n_V", c_int), ("k_R", c_int), ("smooth_pre", c_int), ("smooth_post", c_int),
                ("precision", c_int), ("coarse_max", c_int), ("use_graphs", c_int), ("fuse_coarse", c_int),
                ("tile_fine", c_int), ("use_pdl", c_int), ("reorth", c_int),
                ("gmres_rtol", c_double), ("newton_atol", c_double), ("newton_rtol", c_double),
                ("smooth_lo_frac", c_double)]


class StepInfo(Structure):
    _fields_ = [("newton_its", c_int), ("gmres_its", c_int), ("converged", c_int), ("last_gmres_its", c_int),
                ("rel_resid", c_double), ("newton_resid", c_double), ("newton_resid0", c_double),
                ("solve_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(Structure):
    _fields_ = [("grid", c_void_p), ("u", c_void_p), ("w", c_void_p), ("steps", c_int), ("status", c_int),
                ("newton_its", c_int), ("gmres_its", c_int), ("seconds", c_double)]


class BatchInfo(Structure):
    _fields_ = [("completed", c_int), ("failed", c_int), ("seconds", c_double)]


class ServeRequest(Structure):
    _fields_ = [("dim", c_int), ("n", c_int), ("params", Params), ("opts", POINTER(Opts)), ("u", c_void_p),
                ("w", c_void_p), ("init_w", c_int), ("steps", c_int), ("arrival", c_double), ("status", c_int),
                ("newton_its", c_int), ("gmres_its", c_int), ("t_admit", c_double), ("t_done", c_double),
                ("device_bytes", c_longlong), ("message", ctypes.c_char * 96)]


class ServeInfo(Structure):
    _fields_ = [("completed", c_int), ("failed", c_int), ("peak_inflight", c_int), ("peak_bytes", c_longlong),
                ("seconds", c_double), ("peak_cohort", c_int), ("cohort_steps", c_int)]


class KernelStat(Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("samples", c_longlong), ("total_ms", c_double)]


class OkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) the CUDA library; raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    if build and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; build it with "
                           f"paper_1603_04570_gb300._build.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = c_void_p
    sig = {
        "ok_default_opts": (None, [POINTER(Opts)]),
        "ok_grid_create": (c_int, [c_int, c_int, POINTER(Params), POINTER(Opts), POINTER(c_void_p)]),
        "ok_grid_destroy": (c_int, [P]),
        "ok_grid_query": (c_int, [P, POINTER(c_longlong), POINTER(c_int), POINTER(c_longlong)]),
        "ok_init_w": (c_int, [P, P, P, P]),
        "ok_assemble_rhs": (c_int, [P, P, P, P, P, P, POINTER(c_double), P]),
        "ok_apply_jacobian": (c_int, [P, P, P, P, P]),
        "ok_apply_preconditioner": (c_int, [P, P, P, P, P]),
        "ok_solve_linear": (c_int, [P, P, P, P, POINTER(StepInfo), P]),
        "ok_newton_step": (c_int, [P, P, P, P, P, POINTER(StepInfo), P]),
        "ok_timestep": (c_int, [P, P, P, POINTER(StepInfo), P]),
        "ok_solve_batch": (c_int, [POINTER(Request), c_int, POINTER(BatchInfo), P]),
        "ok_serve": (c_int, [POINTER(ServeRequest), c_int, c_int, c_longlong, POINTER(ServeInfo)]),
        "ok_profile": (c_int, [P, c_int]),
        "ok_profile_read": (c_int, [P, POINTER(KernelStat), c_int, POINTER(c_int)]),
        "ok_launch_count": (c_longlong, []),
        "ok_energy": (c_int, [P, P, P, P, P]),
        "ok_grid_tuning": (c_int, [P, POINTER(c_int), POINTER(c_int), c_int, POINTER(c_int)]),
        "ok_tuning_save": (c_int, [c_char_p]),
        "ok_tuning_load": (c_int, [c_char_p]),
        "ok_apply_jacobian_noalloc": (c_int, [c_int, c_int, POINTER(Params), P, P, P, P]),
        "ok_arnoldi_hessenberg": (c_int, [P, P, c_int, c_int, POINTER(c_int), P]),
        "ok_ritz_values": (c_int, [P, P, P, c_int, POINTER(c_int), P]),
        "ok_givens_unrotate": (c_int, [c_int, P, c_int, P, P]),
        "ok_hessenberg_eigenvalues": (c_int, [c_int, P, c_int, P, P]),
        "ok_last_error": (c_char_p, []),
        "ok_version": (c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(a, n=None, name="array"):
    """Raw pointer of a float64 contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):                    # torch
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float64 tensor")
        if n is not None and a.numel() != n:
            raise ValueError(f"{name} has {a.numel()} entries, expected {n}")
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a contiguous float64 numpy array or torch tensor")
    if n is not None and a.size != n:
        raise ValueError(f"{name} has {a.size} entries, expected {n}")
    return a.ctypes.data


def _stream(stream, *arrays):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    for a in arrays:
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _check(st):
    if st != OK_SUCCESS:
        raise OkError(st, load().ok_last_error().decode())


def ok_default_opts(**overrides) -> Opts:
    o = Opts()
    load().ok_default_opts(byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def ok_grid_create(dim, n, params: Params, opts: Opts | None = None):
    h = c_void_p()
    _check(load().ok_grid_create(dim, n, byref(params), byref(opts) if opts is not None else None, byref(h)))
    return h


def ok_grid_destroy(h):
    _check(load().ok_grid_destroy(h))


def ok_grid_query(h):
    nv, nl, nb = c_longlong(), c_int(), c_longlong()
    _check(load().ok_grid_query(h, byref(nv), byref(nl), byref(nb)))
    return nv.value, nl.value, nb.value


def ok_init_w(h, nv, u0, w0, stream=None):
    _check(load().ok_init_w(h, _ptr(u0, nv, "u0"), _ptr(w0, nv, "w0"), _stream(stream, u0, w0)))


def ok_assemble_rhs(h, nv, u_n, w_n, u_k, w_k, f, stream=None):
    nrm = c_double()
    _check(load().ok_assemble_rhs(h, _ptr(u_n, nv, "u_n"), _ptr(w_n, nv, "w_n"), _ptr(u_k, nv, "u_k"),
                                  _ptr(w_k, nv, "w_k"), _ptr(f, 2 * nv, "f"), byref(nrm),
                                  _stream(stream, f, u_k)))
    return nrm.value


def ok_apply_jacobian(h, nv, u_k, z, y, stream=None):
    _check(load().ok_apply_jacobian(h, _ptr(u_k, nv, "u_k"), _ptr(z, 2 * nv, "z"), _ptr(y, 2 * nv, "y"),
                                    _stream(stream, y, z)))


def ok_apply_preconditioner(h, nv, u_k, v, z, stream=None):
    _check(load().ok_apply_preconditioner(h, _ptr(u_k, nv, "u_k"), _ptr(v, 2 * nv, "v"), _ptr(z, 2 * nv, "z"),
                                          _stream(stream, z, v)))


def _info_call(fn, *args):
    info = StepInfo()
    st = fn(*args[:-1], byref(info), args[-1])
    return st, info


def ok_solve_linear(h, nv, u_k, f, x, stream=None, check=True):
    st, info = _info_call(load().ok_solve_linear, h, _ptr(u_k, nv, "u_k"), _ptr(f, 2 * nv, "f"),
                          _ptr(x, 2 * nv, "x"), _stream(stream, x, f))
    if check:
        _check(st)
    return info


def ok_newton_step(h, nv, u_n, w_n, u_k, w_k, stream=None, check=True):
    st, info = _info_call(load().ok_newton_step, h, _ptr(u_n, nv, "u_n"), _ptr(w_n, nv, "w_n"),
                          _ptr(u_k, nv, "u_k"), _ptr(w_k, nv, "w_k"), _stream(stream, u_k, w_k))
    if check:
        _check(st)
    return info


def ok_timestep(h, nv, u, w, stream=None, check=True):
    st, info = _info_call(load().ok_timestep, h, _ptr(u, nv, "u"), _ptr(w, nv, "w"), _stream(stream, u, w))
    if check:
        _check(st)
    return info


def ok_profile(h, enable: bool):
    _check(load().ok_profile(h, 1 if enable else 0))


def ok_profile_read(h):
    """{kernel class: (samples, total_ms)} of the handle's sampled timings."""
    arr = (KernelStat * 64)()
    n = c_int()
    _check(load().ok_profile_read(h, arr, len(arr), byref(n)))
    return {arr[i].name.decode(): (arr[i].samples, arr[i].total_ms) for i in range(n.value)}


def ok_apply_jacobian_noalloc(dim, n, params: Params, u_k, z, y, stream=None):
    """y = J(u_k) z with no device allocation (device arrays only; see include/ok.h)."""
    nv = (n + 1) ** dim
    _check(load().ok_apply_jacobian_noalloc(dim, n, byref(params), _ptr(u_k, nv, "u_k"), _ptr(z, 2 * nv, "z"),
                                            _ptr(y, 2 * nv, "y"), _stream(stream, y, z)))


def ok_arnoldi_hessenberg(h, max_k=63, stream=None):
    """Hbar ((k+1) x k numpy array) of the handle's last FGMRES restart cycle."""
    import numpy as np
    H = np.zeros((max_k + 1, max(max_k, 1)), order="F")
    k = c_int()
    _check(load().ok_arnoldi_hessenberg(h, H.ctypes.data, max_k + 1, max_k, byref(k), _stream(stream)))
    return np.ascontiguousarray(H[:k.value + 1, :k.value])


def ok_ritz_values(h, limit=63, stream=None):
    """Eigenvalues of the square Arnoldi matrix of the last cycle, at most `limit` steps
    (complex numpy array)."""
    import numpy as np
    re, im = np.zeros(max(limit, 1)), np.zeros(max(limit, 1))
    k = c_int()
    _check(load().ok_ritz_values(h, re.ctypes.data, im.ctypes.data, limit, byref(k), _stream(stream)))
    return re[:k.value] + 1j * im[:k.value]


def _host_status(st, what):
    if st != OK_SUCCESS:
        raise OkError(st, what)


def ok_givens_unrotate(R, cs, sn):
    """The Hessenberg matrix whose Givens reduction (rotations cs, sn) is R ((k+1) x k)."""
    import numpy as np
    k = R.shape[1]
    H = np.array(R, dtype=np.float64, order="F")
    cs, sn = np.ascontiguousarray(cs, dtype=np.float64), np.ascontiguousarray(sn, dtype=np.float64)
    if H.shape != (k + 1, k) or cs.size < k or sn.size < k:
        raise ValueError("R must be (k+1) x k with k rotations")
    _host_status(load().ok_givens_unrotate(k, H.ctypes.data, k + 1, cs.ctypes.data, sn.ctypes.data),
                 "ok_givens_unrotate rejected its arguments")
    return np.ascontiguousarray(H)


def ok_hessenberg_eigenvalues(H):
    """Eigenvalues of a square upper Hessenberg matrix (complex numpy array)."""
    import numpy as np
    A = np.array(H, dtype=np.float64, order="F")
    k = A.shape[0]
    if A.ndim != 2 or A.shape[1] != k:
        raise ValueError("H must be square")
    re, im = np.zeros(max(k, 1)), np.zeros(max(k, 1))
    st = load().ok_hessenberg_eigenvalues(k, A.ctypes.data if k else None, max(k, 1), re.ctypes.data,
                                           im.ctypes.data)
    _host_status(st, {OK_ERR_NONFINITE: "non-finite entry", OK_ERR_NOT_CONVERGED: "QR iteration did not converge"}
                 .get(st, "invalid argument"))
    return re[:k] + 1j * im[:k]


def ok_energy(h, nv, u, stream=None):
    """The Ohta--Kawasaki energy of u: (terms [interfacial, double well, nonlocal], total)."""
    terms = (c_double * 3)()
    total = c_double()
    _check(load().ok_energy(h, _ptr(u, nv, "u"), terms, byref(total), _stream(stream, u)))
    return [terms[0], terms[1], terms[2]], total.value


def ok_grid_tuning(h):
    """[(level cells per side, choice)] the autotuner recorded for the handle."""
    n, c, k = (c_int * 64)(), (c_int * 64)(), c_int()
    _check(load().ok_grid_tuning(h, n, c, 64, byref(k)))
    return [(n[i], c[i]) for i in range(k.value)]


def ok_tuning_save(path: str):
    _check(load().ok_tuning_save(os.fsencode(path)))


def ok_tuning_load(path: str):
    _check(load().ok_tuning_load(os.fsencode(path)))


def ok_launch_count() -> int:
    return load().ok_launch_count()


def ok_solve_batch(requests, stream=None):
    """requests: list of (Grid, u, w, steps).  Returns (status list, BatchInfo)."""
    arr = (Request * len(requests))()
    for i, (g, u, w, steps) in enumerate(requests):
        arr[i].grid = g.handle
        arr[i].u = _ptr(u, g.nv, "u")
        arr[i].w = _ptr(w, g.nv, "w")
        arr[i].steps = steps
    out = BatchInfo()
    st = load().ok_solve_batch(arr, len(requests), byref(out), _stream(stream, *(r[1] for r in requests)))
    return st, [arr[i] for i in range(len(requests))], out


def ok_serve(requests, max_inflight, mem_budget):
    """requests: list of dicts with dim, n, eps, sigma, m, theta, dt, u, w, steps,
    and optionally arrival (s), init_w (bool), opts (dict of ok_opts fields).
    u and w are updated in place.  Returns (status, [ServeRequest], ServeInfo)."""
    arr = (ServeRequest * len(requests))()
    keep = []
    for i, r in enumerate(requests):
        nv = (r["n"] + 1) ** r["dim"]
        q = arr[i]
        q.dim, q.n = r["dim"], r["n"]
        q.params = Params(r["eps"], r["sigma"], r["m"], r["theta"], r["dt"])
        if r.get("opts"):
            o = ok_default_opts(**r["opts"])
            keep.append(o)
            q.opts = ctypes.pointer(o)
        q.u = _ptr(r["u"], nv, "u")
        q.w = _ptr(r["w"], nv, "w")
        q.init_w = 1 if r.get("init_w") else 0
        q.steps = r["steps"]
        q.arrival = float(r.get("arrival", 0.0))
    info = ServeInfo()
    st = load().ok_serve(arr, len(requests), max_inflight, int(mem_budget), byref(info))
    return st, [arr[i] for i in range(len(requests))], info


class Grid:
    """One solver handle (grid + parameters + workspace on the current device)."""

    def __init__(self, dim, n, eps, sigma, m, theta, dt, **opts):
        self.dim, self.n = dim, n
        self.params = Params(eps, sigma, m, theta, dt)
        self.opts = ok_default_opts(**opts)
        self.handle = ok_grid_create(dim, n, self.params, self.opts)
        self.nv, self.levels, self.device_bytes = ok_grid_query(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            ok_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_w(self, u0, w0, stream=None):
        ok_init_w(self.handle, self.nv, u0, w0, stream)

    def assemble_rhs(self, u_n, w_n, u_k, w_k, f, stream=None):
        return ok_assemble_rhs(self.handle, self.nv, u_n, w_n, u_k, w_k, f, stream)

    def apply_jacobian(self, u_k, z, y, stream=None):
        ok_apply_jacobian(self.handle, self.nv, u_k, z, y, stream)

    def apply_preconditioner(self, u_k, v, z, stream=None):
        ok_apply_preconditioner(self.handle, self.nv, u_k, v, z, stream)

    def solve_linear(self, u_k, f, x, stream=None, check=True):
        return ok_solve_linear(self.handle, self.nv, u_k, f, x, stream, check)

    def newton_step(self, u_n, w_n, u_k, w_k, stream=None, check=True):
        return ok_newton_step(self.handle, self.nv, u_n, w_n, u_k, w_k, stream, check)

    def timestep(self, u, w, stream=None, check=True):
        return ok_timestep(self.handle, self.nv, u, w, stream, check)

    def tuning(self):
        return ok_grid_tuning(self.handle)

    def energy(self, u, stream=None):
        return ok_energy(self.handle, self.nv, u, stream)

    def arnoldi_hessenberg(self, max_k=63, stream=None):
        return ok_arnoldi_hessenberg(self.handle, max_k, stream)

    def ritz_values(self, limit=63, stream=None):
        return ok_ritz_values(self.handle, limit, stream)


def version() -> str:
    return load().ok_version().decode()
