"""FP64 CPU oracle of the DDLR preconditioner -- TEST INFRASTRUCTURE ONLY.

The oracle is the correctness reference that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product package never does, and the two
share no code.  The arithmetic lives in ``ddlr_oracle.c`` (plain C, FP64,
following the paper's steps in order); this module compiles it with gcc and
marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddlr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libddlr_oracle.so")

STATUS = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "BREAKDOWN", 4: "NOT_SPD",
          5: "NOCONV"}


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle {where}: {STATUS.get(code, code)}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no -march)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                           "-fno-fast-math", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.or_setup.argtypes = [I, P, P, P, P, I, I, I, D, I, I, I, I, I, I, I, D,
                                 ctypes.c_ulonglong, I, I, I, I, I, I, I, I, D, I, I, I, ctypes.POINTER(P)]
        lib.or_setup.restype = I
        lib.or_destroy.argtypes = [P]
        lib.or_apply.argtypes = [P, P, P]
        lib.or_apply.restype = I
        lib.or_a0_solve.argtypes = [P, P, P]
        lib.or_a0_solve.restype = I
        lib.or_pcg.argtypes = [P, P, P, D, I, I, ctypes.POINTER(I),
                               ctypes.POINTER(D)]
        lib.or_pcg.restype = I
        lib.or_gmres.argtypes = [P, P, P, D, I, I, ctypes.POINTER(I), ctypes.POINTER(D)]
        lib.or_gmres.restype = I
        lib.or_info.argtypes = [P, P, ctypes.POINTER(D)]
        lib.or_ritz.argtypes = [P, P]
        lib.or_perm.argtypes = [P, P]
        lib.or_lowrank.argtypes = [P, P, P, P]
        lib.or_factor_nnz.argtypes = [P]
        lib.or_factor_nnz.restype = ctypes.c_long
        lib.or_factor_coo.argtypes = [P, P, P, P]
        lib.or_cheb_bounds.argtypes = [P, P]
        lib.or_set_cheb_bounds.argtypes = [P, D, D]
        lib.or_reorth_passes.argtypes = [P]
        lib.or_reorth_passes.restype = ctypes.c_long
        lib.or_sm64_pm1.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong]
        lib.or_sm64_pm1.restype = D
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def sm64_pm1(seed: int, i: int) -> float:
    return _load().or_sm64_pm1(seed, i)


class Oracle:
    """DDLR setup + apply + PCG in FP64 on the CPU.

    ``A = (n, rowptr, colind, val)`` full symmetric CSR, ``part[i]`` in [0, p).
    Options follow the library's: variant 1/2, rank k, alpha, theta_mode
    (1: theta = Ritz_{k+1}, 0: theta = 0), factor (0: IC(0), 1: exact
    Cholesky, 2: incomplete LDL^T on the pattern, 3: exact LDL^T),
    fill_level (incomplete factors: the level of fill of their pattern, 0 =
    the pattern of A0),
    c_order (0: ascending index, 1: greedy multicolour) of C_a, b_order (the
    same choice for the interior blocks), scale_diag,
    lanczos_max (0: 5k), lanczos_check (10), lanczos_eps (1e-4), seed,
    c_solver (0: C_a factored; 1: Chebyshev with block Jacobi, Sec. 4.3),
    cheb_steps (5) and cheb_lanczos (20, steps of the spectrum estimate),
    lowrank_method (0: Lanczos; 1: randomized subspace iteration with
    ell = k + rand_oversample columns and rand_power power steps; 2: Lanczos
    bidiagonalisation of A0^-1 E, DDLR-2 only),
    c_solver 2 = MR approximate inverse of C_a (Algorithm 2) with mr_iters
    iterations, at most mr_lfil entries per column of Z and drop tolerance
    mr_droptol relative to the column norm.  indefinite=1 accepts a
    preconditioner that is not SPD (Ritz values >= 1 for DDLR-1, an
    indefinite I - K for DDLR-2) for use with GMRES.  lanczos_reorth: 0 = a
    second Gram-Schmidt pass only when the first shrank the Lanczos vector
    below 1/sqrt(2) of its norm, 1 = always two passes.
    """

    def __init__(self, A, part, p, *, variant=1, k=8, alpha=1.0, theta_mode=1,
                 factor=0, c_order=0, b_order=0, scale_diag=0, lanczos_max=0,
                 lanczos_check=10, lanczos_eps=1e-4, seed=0, c_solver=0,
                 cheb_steps=5, cheb_lanczos=20, lowrank_method=0, rand_oversample=10,
                 rand_power=2, mr_iters=3, mr_lfil=6, mr_droptol=1e-3, indefinite=0, fill_level=0,
                 lanczos_reorth=0):
        lib = _load()
        n, rp, ci, va = A
        self._keep = [np.ascontiguousarray(rp, dtype=np.int32),
                      np.ascontiguousarray(ci, dtype=np.int32),
                      np.ascontiguousarray(va, dtype=np.float64),
                      np.ascontiguousarray(part, dtype=np.int32)]
        h = ctypes.c_void_p()
        st = lib.or_setup(int(n), *[_ptr(a) for a in self._keep], int(p),
                          int(variant), int(k), float(alpha), int(theta_mode),
                          int(factor), int(c_order), int(b_order), int(scale_diag),
                          int(lanczos_max), int(lanczos_check),
                          float(lanczos_eps), int(seed), int(c_solver),
                          int(cheb_steps), int(cheb_lanczos), int(lowrank_method),
                          int(rand_oversample), int(rand_power), int(mr_iters), int(mr_lfil),
                          float(mr_droptol), int(indefinite), int(fill_level), int(lanczos_reorth),
                          ctypes.byref(h))
        if st != 0:
            raise OracleError(st, "setup")
        self._h = h
        info = np.zeros(9, dtype=np.int32)
        th = ctypes.c_double()
        lib.or_info(h, _ptr(info), ctypes.byref(th))
        (self.n, self.p, self.s, self.m, self.k, self.msteps, self.ncolors,
         self.variant, self.urows) = [int(v) for v in info]
        self.theta = th.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    @property
    def cheb_bounds(self):
        """(lo, hi): the spectrum interval of the Chebyshev C_a solve"""
        b = np.empty(2)
        _load().or_cheb_bounds(self._h, _ptr(b))
        return float(b[0]), float(b[1])

    def set_cheb_bounds(self, lo, hi):
        """Replace the Chebyshev interval (the setup's low-rank data stay)."""
        _load().or_set_cheb_bounds(self._h, float(lo), float(hi))

    def apply(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        _load().or_apply(self._h, _ptr(x), _ptr(y))
        return y

    def a0_solve(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        _load().or_a0_solve(self._h, _ptr(x), _ptr(y))
        return y

    def pcg(self, b, tol=1e-8, maxit=500, flexible=False):
        """Returns (x, its, true_relres, status)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        its = ctypes.c_int()
        rel = ctypes.c_double()
        st = _load().or_pcg(self._h, _ptr(b), _ptr(x), float(tol), int(maxit),
                            int(bool(flexible)), ctypes.byref(its),
                            ctypes.byref(rel))
        return x, its.value, rel.value, STATUS.get(st, st)

    def gmres(self, b, tol=1e-8, maxit=500, restart=40):
        """Right-preconditioned GMRES(restart) from x0 = 0.
        Returns (x, its, true_relres, status)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        its = ctypes.c_int()
        rel = ctypes.c_double()
        st = _load().or_gmres(self._h, _ptr(b), _ptr(x), float(tol), int(maxit), int(restart),
                              ctypes.byref(its), ctypes.byref(rel))
        return x, its.value, rel.value, STATUS.get(st, st)

    @property
    def reorth_passes(self):
        """Gram-Schmidt passes taken by the Lanczos steps of the setup"""
        return int(_load().or_reorth_passes(self._h))

    @property
    def ritz(self):
        r = np.empty(self.msteps)
        _load().or_ritz(self._h, _ptr(r))
        return r

    @property
    def perm(self):
        """new index (eq. Bmat order) -> original index"""
        q = np.empty(self.n, dtype=np.int32)
        _load().or_perm(self._h, _ptr(q))
        return q

    def lowrank(self):
        """(U, lam, Hk): U has ``urows`` rows in eq. Bmat order (interface rows
        only for DDLR-1, all rows for DDLR-2), lam = Lambda_k (DDLR-1) and
        Hk (DDLR-2); missing parts are None."""
        U = np.empty((self.urows, self.k))
        lam = np.empty(self.k)
        Hk = np.empty((self.k, self.k))
        _load().or_lowrank(self._h, _ptr(U), _ptr(lam), _ptr(Hk))
        if self.variant == 1:
            return U, lam, None
        return U, None, Hk

    def lowrank_original_order(self):
        """U with rows indexed by ascending original index of the rows it
        covers (interface nodes for DDLR-1, all nodes for DDLR-2)."""
        U, lam, Hk = self.lowrank()
        perm = self.perm
        rows = perm[self.m:] if self.variant == 1 else perm
        order = np.argsort(rows, kind="stable")
        return U[order], lam, Hk, np.sort(rows)

    def factor_coo(self):
        """All local factor entries (lower, incl. diagonal) as (row, col, val)
        in original indices."""
        lib = _load()
        nnz = lib.or_factor_nnz(self._h)
        r = np.empty(nnz, dtype=np.int32)
        c = np.empty(nnz, dtype=np.int32)
        v = np.empty(nnz)
        lib.or_factor_coo(self._h, _ptr(r), _ptr(c), _ptr(v))
        return r, c, v
