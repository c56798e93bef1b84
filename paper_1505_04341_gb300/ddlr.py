"""Thin ctypes binding of the DDLR C ABI (include/ddlr.h).

Argument marshalling only: every step of setup, apply and solve runs in the
CUDA library.  Vectors may be torch CUDA tensors (device memory, the call is
issued on the tensor's current stream) or numpy arrays (host memory, staged by
the library).  The library must be built (``build.build()``); a missing library
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "BREAKDOWN", 4: "NOT_SPD",
          5: "NOCONV", 6: "TIMEOUT", 7: "NAN", 8: "CUDA"}


class DdlrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class ddlr_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("rank_k", ctypes.c_int),
                ("alpha", ctypes.c_double), ("theta_mode", ctypes.c_int),
                ("factor", ctypes.c_int), ("c_order", ctypes.c_int),
                ("b_order", ctypes.c_int),
                ("precision", ctypes.c_int), ("uk_bf16", ctypes.c_int),
                ("scale_diag", ctypes.c_int), ("lanczos_max", ctypes.c_int),
                ("lanczos_check", ctypes.c_int), ("lanczos_eps", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("max_nrhs", ctypes.c_int),
                ("c_solver", ctypes.c_int), ("cheb_steps", ctypes.c_int),
                ("cheb_lanczos", ctypes.c_int), ("lowrank_method", ctypes.c_int),
                ("rand_oversample", ctypes.c_int), ("rand_power", ctypes.c_int),
                ("mr_iters", ctypes.c_int), ("mr_lfil", ctypes.c_int), ("mr_droptol", ctypes.c_double),
                ("indefinite", ctypes.c_int), ("fill_level", ctypes.c_int),
                ("lanczos_reorth", ctypes.c_int), ("wait_limit_s", ctypes.c_double)]


class ddlr_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("p", ctypes.c_int), ("s", ctypes.c_int),
                ("m", ctypes.c_int), ("k", ctypes.c_int), ("variant", ctypes.c_int),
                ("precision", ctypes.c_int), ("lanczos_steps", ctypes.c_int),
                ("ncolors", ctypes.c_int), ("levels_interior", ctypes.c_int),
                ("levels_c", ctypes.c_int), ("theta", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("nnz_a", ctypes.c_longlong),
                ("nnz_factor", ctypes.c_longlong), ("nnz_ehat", ctypes.c_longlong),
                ("fill_ratio", ctypes.c_double), ("device_bytes", ctypes.c_longlong),
                ("setup_ms", ctypes.c_double), ("batch_block_chunks", ctypes.c_int),
                ("batch_block_elem", ctypes.c_int), ("plan_ms", ctypes.c_double),
                ("persistent", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("cheb_lanczos_steps", ctypes.c_int),
                ("reorth_passes", ctypes.c_int), ("reorth_fp32", ctypes.c_int)]


class ddlr_solve_info(ctypes.Structure):
    _fields_ = [("its", ctypes.c_int), ("relres", ctypes.c_double),
                ("status", ctypes.c_int)]


class ddlr_server_options(ctypes.Structure):
    _fields_ = [("max_concurrent", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("memory_fraction", ctypes.c_double)]


# every entry point declared in include/ddlr.h
EXPORTS = ["ddlr_options_default", "ddlr_setup", "ddlr_refactor", "ddlr_apply",
           "ddlr_a0_solve", "ddlr_a0_solve_noalloc", "ddlr_pcg", "ddlr_gmres", "ddlr_increase_rank", "ddlr_get_info", "ddlr_get_ritz",
           "ddlr_get_factor_coo", "ddlr_get_lowrank", "ddlr_set_lowrank", "ddlr_set_cheb_bounds",
           "ddlr_set_timing", "ddlr_get_counters", "ddlr_reset_counters",
           "ddlr_get_traffic", "ddlr_set_stream", "ddlr_set_wait_limit", "ddlr_selftest_conversions",
           "ddlr_last_error",
           "ddlr_destroy", "ddlr_server_options_default", "ddlr_server_create",
           "ddlr_server_add_model", "ddlr_server_submit", "ddlr_server_wait",
           "ddlr_server_stats", "ddlr_server_last_error", "ddlr_server_destroy"]

_lib = None


def load(path: str | None = None):
    """Load the built library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"DDLR CUDA library not built ({path}); run "
                           "paper_1505_04341_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    LL = ctypes.c_longlong
    sig = {
        "ddlr_options_default": ([ctypes.POINTER(ddlr_options)], I),
        "ddlr_setup": ([I, P, P, P, P, I, ctypes.POINTER(ddlr_options), P,
                        ctypes.POINTER(P)], I),
        "ddlr_refactor": ([P, P], I),
        "ddlr_increase_rank": ([P, I], I),
        "ddlr_apply": ([P, P, P, I, I], I),
        "ddlr_a0_solve": ([P, P, P, I, I], I),
        "ddlr_a0_solve_noalloc": ([P, P, P], I),
        "ddlr_pcg": ([P, P, P, I, I, D, I, ctypes.POINTER(ddlr_solve_info)], I),
        "ddlr_gmres": ([P, P, P, D, I, I, ctypes.POINTER(ddlr_solve_info)], I),
        "ddlr_get_info": ([P, ctypes.POINTER(ddlr_info)], I),
        "ddlr_get_ritz": ([P, P, I, ctypes.POINTER(I)], I),
        "ddlr_get_factor_coo": ([P, ctypes.POINTER(LL), P, P, P], I),
        "ddlr_get_lowrank": ([P, P, P, P, P], I),
        "ddlr_set_lowrank": ([P, P, P, D, P], I),
        "ddlr_set_cheb_bounds": ([P, D, D], I),
        "ddlr_set_timing": ([P, I], I),
        "ddlr_get_counters": ([P, ctypes.POINTER(LL), ctypes.c_char_p, I, P, P,
                               I, ctypes.POINTER(I)], I),
        "ddlr_reset_counters": ([P], I),
        "ddlr_get_traffic": ([P, P, P, P, I], I),
        "ddlr_set_stream": ([P, P], I),
        "ddlr_set_wait_limit": ([P, D], I),
        "ddlr_selftest_conversions": ([P, LL, I, ctypes.POINTER(LL)], I),
        "ddlr_last_error": ([P], ctypes.c_char_p),
        "ddlr_destroy": ([P], I),
        "ddlr_server_options_default": ([ctypes.POINTER(ddlr_server_options)], I),
        "ddlr_server_create": ([ctypes.POINTER(ddlr_server_options), ctypes.POINTER(P)], I),
        "ddlr_server_add_model": ([P, I, P, P, P, P, I, ctypes.POINTER(ddlr_options),
                                   ctypes.POINTER(I)], I),
        "ddlr_server_submit": ([P, I, P, ctypes.POINTER(LL)], I),
        "ddlr_server_wait": ([P, LL, D, P, ctypes.POINTER(ddlr_solve_info),
                              ctypes.POINTER(D), ctypes.POINTER(I)], I),
        "ddlr_server_stats": ([P, ctypes.POINTER(LL), ctypes.POINTER(I), ctypes.POINTER(I),
                               ctypes.POINTER(I), ctypes.POINTER(LL)], I),
        "ddlr_server_last_error": ([P], ctypes.c_char_p),
        "ddlr_server_destroy": ([P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _vec_ptr(v):
    """(pointer, n, ncols, is_device) of a float64 vector or column-major block."""
    if isinstance(v, np.ndarray):
        if v.dtype != np.float64:
            raise TypeError("float64 required")
        if v.ndim == 2 and not v.flags.f_contiguous:
            raise TypeError("2-D arrays must be column-major (Fortran order)")
        if v.ndim == 1 and not v.flags.c_contiguous:
            raise TypeError("contiguous array required")
        return ctypes.c_void_p(v.ctypes.data), v.shape[0], (v.shape[1] if v.ndim == 2 else 1)
    import torch
    if not isinstance(v, torch.Tensor) or v.dtype != torch.float64:
        raise TypeError("float64 numpy array or torch tensor required")
    if v.dim() == 2:
        # column-major n x nrhs == row-major (nrhs, n) storage
        if v.stride(0) != 1 or v.stride(1) != v.shape[0]:
            raise TypeError("2-D tensors must be column-major (use t.T.contiguous().T)")
        return ctypes.c_void_p(v.data_ptr()), v.shape[0], v.shape[1]
    if not v.is_contiguous():
        raise TypeError("contiguous tensor required")
    return ctypes.c_void_p(v.data_ptr()), v.shape[0], 1


def selftest_conversions(values, direction: int) -> int:
    """Mismatches of the library's bit-pattern binary64 <-> binary32
    conversions against the device's (values: a CUDA float64 tensor; direction
    0 narrows, 1 widens the low 32 bits read as binary32)."""
    lib = load()
    ptr, n, _ = _vec_ptr(values)
    bad = ctypes.c_longlong(0)
    _check(lib, None, lib.ddlr_selftest_conversions(ptr, n, int(direction), ctypes.byref(bad)))
    return bad.value


def _check(lib, h, st):
    if st != 0:
        msg = lib.ddlr_last_error(h)
        raise DdlrError(st, msg.decode() if msg else "")


def options(**kw) -> ddlr_options:
    lib = load()
    o = ddlr_options()
    lib.ddlr_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class DDLR:
    """Handle of a built DDLR preconditioner (see include/ddlr.h)."""

    def __init__(self, A, part, p, stream=None, **opts):
        lib = load()
        n, rp, ci, va = A
        self._arrays = [np.ascontiguousarray(rp, dtype=np.int32),
                        np.ascontiguousarray(ci, dtype=np.int32),
                        np.ascontiguousarray(va, dtype=np.float64),
                        np.ascontiguousarray(part, dtype=np.int32)]
        self.opts = options(**opts)
        h = ctypes.c_void_p()
        st = lib.ddlr_setup(int(n), *[_np_ptr(a) for a in self._arrays], int(p),
                            ctypes.byref(self.opts), self._stream_ptr(stream),
                            ctypes.byref(h))
        _check(lib, None, st)
        self._h = h
        self.n = int(n)
        self.nnz = int(len(ci))

    @staticmethod
    def _stream_ptr(stream):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            except ImportError:
                pass
            return ctypes.c_void_p(0)
        if isinstance(stream, int):
            return ctypes.c_void_p(stream)
        return ctypes.c_void_p(stream.cuda_stream)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.ddlr_destroy(self._h)
            self._h = None

    __del__ = close

    def set_wait_limit(self, seconds):
        """Limit of the handle's bounded device waits (seconds)."""
        _check(_lib, self._h, _lib.ddlr_set_wait_limit(self._h, float(seconds)))

    def set_stream(self, stream):
        _check(_lib, self._h, _lib.ddlr_set_stream(self._h, self._stream_ptr(stream)))

    def increase_rank(self, k_new: int):
        """Raise the rank to k_new, continuing the Lanczos process (Sec. 3.4)."""
        _check(_lib, self._h, _lib.ddlr_increase_rank(self._h, int(k_new)))

    def refactor(self, val=None):
        ptr = None
        if val is not None:
            ptr = _vec_ptr(val)[0]
        _check(_lib, self._h, _lib.ddlr_refactor(self._h, ptr))

    def _vec_op(self, fn, x, y):
        px, n, nr = _vec_ptr(x)
        py, n2, nr2 = _vec_ptr(y)
        if n != self.n or n2 != self.n or nr != nr2:
            raise ValueError("shape mismatch")
        _check(_lib, self._h, fn(self._h, px, py, nr, n))
        return y

    def _like(self, x):
        if isinstance(x, np.ndarray):
            return np.zeros_like(x, order="F")
        import torch
        return torch.zeros_like(x) if x.dim() == 1 else torch.zeros_like(x.T).T

    def apply(self, x, y=None):
        """y = M^-1 x"""
        return self._vec_op(_lib.ddlr_apply, x, self._like(x) if y is None else y)

    def a0_solve(self, x, y=None):
        """y = A0^-1 x"""
        return self._vec_op(_lib.ddlr_a0_solve, x, self._like(x) if y is None else y)

    def a0_solve_noalloc(self, x, y):
        """y = A0^-1 x for device float64 vectors of length n, through the
        entry point that allocates no device memory (temporaries in a static
        device array; n <= 1,048,576, FP64 handles)."""
        px, n, nr = _vec_ptr(x)
        py, n2, nr2 = _vec_ptr(y)
        if n != self.n or n2 != self.n or nr != 1 or nr2 != 1:
            raise ValueError("shape mismatch: one vector of length n expected")
        _check(_lib, self._h, _lib.ddlr_a0_solve_noalloc(self._h, px, py))
        return y

    def pcg(self, b, x=None, tol=1e-8, maxit=500, check=True):
        """Returns (x, [ddlr_solve_info per RHS]); raises on NOCONV/NAN when
        check is true."""
        x = self._like(b) if x is None else x
        pb, n, nr = _vec_ptr(b)
        px, _, _ = _vec_ptr(x)
        infos = (ddlr_solve_info * nr)()
        st = _lib.ddlr_pcg(self._h, pb, px, nr, n, float(tol), int(maxit), infos)
        if st not in (0, 5, 7) or (check and st != 0):
            _check(_lib, self._h, st)
        return x, [dict(its=i.its, relres=i.relres, status=STATUS[i.status]) for i in infos]

    def gmres(self, b, x=None, tol=1e-8, maxit=500, restart=40, check=True):
        """Right-preconditioned GMRES(restart) from x0 = 0 (one RHS).  Returns
        (x, ddlr_solve_info as a dict); raises on NOCONV/NAN when check is
        true."""
        x = self._like(b) if x is None else x
        pb, n, nr = _vec_ptr(b)
        px, n2, nr2 = _vec_ptr(x)
        if n != self.n or n2 != self.n or nr != 1 or nr2 != 1:
            raise ValueError("shape mismatch: one vector of length n expected")
        inf = ddlr_solve_info()
        st = _lib.ddlr_gmres(self._h, pb, px, float(tol), int(maxit), int(restart), ctypes.byref(inf))
        if st not in (0, 5, 7) or (check and st != 0):
            _check(_lib, self._h, st)
        return x, dict(its=inf.its, relres=inf.relres, status=STATUS[inf.status])

    def info(self) -> dict:
        inf = ddlr_info()
        _check(_lib, self._h, _lib.ddlr_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in ddlr_info._fields_}

    def ritz(self) -> np.ndarray:
        cnt = ctypes.c_int()
        _lib.ddlr_get_ritz(self._h, None, 0, ctypes.byref(cnt))
        out = np.zeros(cnt.value)
        _check(_lib, self._h, _lib.ddlr_get_ritz(self._h, _np_ptr(out), cnt.value, ctypes.byref(cnt)))
        return out

    def factor_coo(self):
        nnz = ctypes.c_longlong()
        _check(_lib, self._h, _lib.ddlr_get_factor_coo(self._h, ctypes.byref(nnz), None, None, None))
        r = np.zeros(nnz.value, np.int32)
        c = np.zeros(nnz.value, np.int32)
        v = np.zeros(nnz.value)
        _check(_lib, self._h, _lib.ddlr_get_factor_coo(self._h, ctypes.byref(nnz), _np_ptr(r), _np_ptr(c), _np_ptr(v)))
        return r, c, v

    def lowrank(self):
        inf = self.info()
        k = inf["k"]
        rows = inf["s"] if inf["variant"] == 1 else inf["n"]
        U = np.zeros((rows, k))
        lam = np.zeros(k)
        th = ctypes.c_double()
        Hk = np.zeros((k, k))
        _check(_lib, self._h, _lib.ddlr_get_lowrank(self._h, _np_ptr(U), _np_ptr(lam), ctypes.byref(th), _np_ptr(Hk)))
        return U, lam, th.value, Hk

    def set_lowrank(self, U, lam=None, theta=0.0, Hk=None):
        U = np.ascontiguousarray(U, dtype=np.float64)
        lam = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
        Hk = None if Hk is None else np.ascontiguousarray(Hk, dtype=np.float64)
        _check(_lib, self._h, _lib.ddlr_set_lowrank(
            self._h, _np_ptr(U), None if lam is None else _np_ptr(lam), float(theta),
            None if Hk is None else _np_ptr(Hk)))

    def set_cheb_bounds(self, lo, hi):
        """Spectrum interval of D_a^-1 C_a for the Chebyshev C_a solve
        (c_solver=1, Sec. 4.3)."""
        _check(_lib, self._h, _lib.ddlr_set_cheb_bounds(self._h, float(lo), float(hi)))

    def set_timing(self, on=True):
        _check(_lib, self._h, _lib.ddlr_set_timing(self._h, int(bool(on))))

    def reset_counters(self):
        _check(_lib, self._h, _lib.ddlr_reset_counters(self._h))

    def counters(self) -> dict:
        L = ctypes.c_longlong()
        nf = ctypes.c_int()
        buf = ctypes.create_string_buffer(4096)
        ms = np.zeros(64)
        cnt = np.zeros(64, np.int64)
        _check(_lib, self._h, _lib.ddlr_get_counters(self._h, ctypes.byref(L), buf, 4096, _np_ptr(ms), _np_ptr(cnt), 64, ctypes.byref(nf)))
        names = buf.value.decode().split(",") if buf.value else []
        fam = {nm: dict(ms=float(ms[i]), launches=int(cnt[i])) for i, nm in enumerate(names)}
        return dict(launches=int(L.value), families=fam)

    def traffic(self) -> dict:
        """Algorithmic bytes of one apply / A0 solve and per launch of each
        kernel family (names as in counters())."""
        a, b = ctypes.c_double(), ctypes.c_double()
        fam = np.zeros(64)
        _check(_lib, self._h, _lib.ddlr_get_traffic(self._h, ctypes.byref(a), ctypes.byref(b), _np_ptr(fam), 64))
        names = list(self.counters()["families"].keys())
        return dict(apply_bytes=a.value, a0_bytes=b.value,
                    family_bytes={nm: float(fam[i]) for i, nm in enumerate(names)})


class Server:
    """Solve service (include/ddlr.h, serving section): resident models,
    continuous batching (slots admitted and retired between iterations),
    admission by device memory."""

    def __init__(self, max_concurrent=8, max_batch=16, tol=1e-8, maxit=500,
                 memory_fraction=0.9):
        lib = load()
        o = ddlr_server_options()
        lib.ddlr_server_options_default(ctypes.byref(o))
        o.max_concurrent, o.max_batch, o.tol, o.maxit, o.memory_fraction = (
            max_concurrent, max_batch, tol, maxit, memory_fraction)
        h = ctypes.c_void_p()
        st = lib.ddlr_server_create(ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            raise DdlrError(st, "server_create")
        self._h = h
        self._n = []

    def _err(self, st):
        if st != 0:
            raise DdlrError(st, _lib.ddlr_server_last_error(self._h).decode())

    def add_model(self, A, part, p, **opts) -> int:
        n, rp, ci, va = A
        arrs = [np.ascontiguousarray(rp, dtype=np.int32), np.ascontiguousarray(ci, dtype=np.int32),
                np.ascontiguousarray(va, dtype=np.float64), np.ascontiguousarray(part, dtype=np.int32)]
        o = options(**opts)
        m = ctypes.c_int()
        self._err(_lib.ddlr_server_add_model(self._h, int(n), *[_np_ptr(a) for a in arrs], int(p),
                                             ctypes.byref(o), ctypes.byref(m)))
        self._n.append(int(n))
        return m.value

    def submit(self, model, b) -> int:
        b = np.ascontiguousarray(b, dtype=np.float64)
        rid = ctypes.c_longlong()
        self._err(_lib.ddlr_server_submit(self._h, int(model), _np_ptr(b), ctypes.byref(rid)))
        return rid.value

    def wait(self, request, n, timeout=0.0):
        """Returns (x, info dict, latency seconds, batch width)."""
        x = np.empty(n)
        info = ddlr_solve_info()
        lat = ctypes.c_double()
        bw = ctypes.c_int()
        st = _lib.ddlr_server_wait(self._h, int(request), float(timeout), _np_ptr(x),
                                   ctypes.byref(info), ctypes.byref(lat), ctypes.byref(bw))
        if st not in (0, 5, 7):
            self._err(st)
        return x, dict(its=info.its, relres=info.relres, status=STATUS[info.status]), lat.value, bw.value

    def stats(self) -> dict:
        c, ar = ctypes.c_longlong(), ctypes.c_longlong()
        mb, mi, nm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._err(_lib.ddlr_server_stats(self._h, ctypes.byref(c), ctypes.byref(mb), ctypes.byref(mi),
                                         ctypes.byref(nm), ctypes.byref(ar)))
        return dict(completed=c.value, max_batch_seen=mb.value, max_inflight_seen=mi.value,
                    models=nm.value, admitted_running=ar.value)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.ddlr_server_destroy(self._h)
            self._h = None

    __del__ = close
