"""Host-side checks of the C ABI library (no GPU needed): the shared library
loads and exports every entry point that include/ddlr.h declares, the option
defaults are the paper's (Sec. 5), and host-side validation rejects bad input
before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1505_04341_gb300 as pkg
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load()


def test_exports_match_header(lib):
    hdr = open(os.path.join(ROOT, "include", "ddlr.h")).read()
    declared = set(re.findall(r"\b(ddlr_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(pkg.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_option_defaults(lib):
    o = pkg.options()
    assert (o.variant, o.rank_k, o.alpha, o.theta_mode) == (1, 16, 1.0, 1)
    assert (o.lanczos_max, o.lanczos_check, o.lanczos_eps) == (0, 10, 1e-4)
    assert (o.factor, o.c_order, o.b_order, o.precision, o.max_nrhs) == (0, 0, 0, 0, 1)


def _setup_status(lib, A, part, p, **kw):
    n, rp, ci, va = A
    arrs = [np.ascontiguousarray(a, dtype=d) for a, d in
            ((rp, np.int32), (ci, np.int32), (va, np.float64), (part, np.int32))]
    o = pkg.options(**kw)
    h = ctypes.c_void_p()
    st = lib.ddlr_setup(int(n), *[ctypes.c_void_p(a.ctypes.data) for a in arrs], int(p),
                        ctypes.byref(o), None, ctypes.byref(h))
    msg = lib.ddlr_last_error(None).decode()
    if st == 0:
        lib.ddlr_destroy(h)
    return st, msg


def test_setup_rejects_bad_input_on_host(lib):
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    n, rp, ci, va = A
    va2 = va.copy()
    va2[1] += 1.0
    st, msg = _setup_status(lib, (n, rp, ci, va2), part, p, rank_k=2)
    assert st == 1 and "symmetric" in msg
    ci2 = ci.copy()
    ci2[0], ci2[1] = ci2[1], ci2[0]
    st, msg = _setup_status(lib, (n, rp, ci2, va), part, p, rank_k=2)
    assert st == 1 and "ascending" in msg
    bad = part.copy()
    bad[3] = 7
    st, msg = _setup_status(lib, A, bad, p, rank_k=2)
    assert st == 1 and "part" in msg
    st, msg = _setup_status(lib, A, part, p, rank_k=10 ** 4)
    assert st == 1
    st, msg = _setup_status(lib, A, np.zeros(n, np.int32), 1, rank_k=2)
    assert st == 1 and "interface" in msg
    st, msg = _setup_status(lib, A, part, p, rank_k=2, variant=3)
    assert st == 1


def test_null_handle_calls(lib):
    assert lib.ddlr_destroy(None) == 0
    assert lib.ddlr_apply(None, None, None, 1, 1) == 1
    assert lib.ddlr_get_info(None, None) == 1


def test_setup_rejects_bad_option_combinations_on_host(lib):
    """Option validation runs before any device work: the values and the
    combinations the library does not serve are INVALID (status 1)."""
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    for kw in (dict(factor=4), dict(factor=-1), dict(factor=2, precision=1), dict(factor=3, c_solver=1),
               dict(factor=2, c_solver=2), dict(factor=3, lowrank_method=1), dict(indefinite=2),
               dict(lowrank_method=2, variant=1), dict(lowrank_method=3), dict(c_solver=3),
               dict(c_solver=2, mr_iters=4, mr_lfil=8), dict(c_solver=1, cheb_steps=0),
               dict(lowrank_method=1, rand_oversample=-1), dict(precision=2), dict(alpha=0.0)):
        st, msg = _setup_status(lib, A, part, p, rank_k=2, **kw)
        assert st == 1, kw


def test_gmres_entry_point_rejects_null_handle(lib):
    assert lib.ddlr_gmres(None, None, None, 1e-8, 10, 40, None) == 1
