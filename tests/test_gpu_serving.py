"""GPU: the solve service (continuous batching across requests and models).

A model's worker runs a block PCG whose columns are slots; converged columns
are handed back and queued requests admitted between iterations.  A request
admitted into a running block gives the same bits as the same request solved
alone, every served result meets the tolerance, and each agrees with the
FP64 oracle's PCG (iterations within one, solution within 1e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MC = dict(c_order=1, b_order=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


def _problem(shape, parts):
    A = W.laplacian(shape)
    part, p = W.box_partition(shape, parts)
    return A, part, p


def test_admitted_mid_block_equals_alone_and_oracle():
    srv = pkg.Server(max_concurrent=3, max_batch=4, tol=1e-8)
    A0, part0, p0 = _problem((16, 16, 16), (2, 2, 2))
    A1, part1, p1 = _problem((24, 20, 18), (3, 2, 2))
    m0 = srv.add_model(A0, part0, p0, rank_k=8, **MC)
    m1 = srv.add_model(A1, part1, p1, rank_k=8, **MC)
    b0 = W.rhs(A0[0], 5)
    x_alone, inf, _, bw = srv.wait(srv.submit(m0, b0), A0[0])
    assert inf["status"] == "OK" and inf["relres"] <= 1e-8 and bw == 1
    # fill model 0's block (4 slots), queue more behind it, then the same
    # request again: it is admitted when a slot frees, into a running block
    ids = []
    for i in range(6):
        ids.append((m0, A0, srv.submit(m0, W.rhs(A0[0], 200 + i))))
        ids.append((m1, A1, srv.submit(m1, W.rhs(A1[0], 100 + i))))
    ids.append((m0, A0, srv.submit(m0, b0)))
    mark = len(ids) - 1
    for i in range(3):
        ids.append((m0, A0, srv.submit(m0, W.rhs(A0[0], 300 + i))))
    res = [srv.wait(r, A[0]) for (_, A, r) in ids]
    st = srv.stats()
    assert st["admitted_running"] > 0                       # admissions into running blocks
    assert st["max_batch_seen"] > 1
    x_mix, inf_mix, _, _ = res[mark]
    assert inf_mix["status"] == "OK"
    assert np.array_equal(x_alone, x_mix)                   # same bits alone and in the mix
    assert inf_mix["its"] == inf["its"]
    # every served result against the oracle's PCG
    orcs = {m0: O.Oracle(A0, part0, p0, k=8, **MC), m1: O.Oracle(A1, part1, p1, k=8, **MC)}
    seeds = []
    for i in range(6):
        seeds += [(m0, 200 + i), (m1, 100 + i)]
    seeds += [(m0, None)] + [(m0, 300 + i) for i in range(3)]
    for (m, seed), (x, info, lat, bw) in zip(seeds, res):
        A = A0 if m == m0 else A1
        b = b0 if seed is None else W.rhs(A[0], seed)
        xo, its_o, rel_o, sto = orcs[m].pcg(b, 1e-8)
        assert sto == "OK" and info["status"] == "OK" and info["relres"] <= 1e-8
        assert abs(info["its"] - its_o) <= 1, (info, its_o)
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
        assert lat > 0 and 1 <= bw <= 4
    srv.close()


def test_widening_keeps_running_columns():
    """A block opened for one request is widened when more arrive while it
    runs; the first request's result is still bitwise its result alone."""
    A, part, p = _problem((20, 20, 20), (2, 2, 2))
    srv = pkg.Server(max_concurrent=1, max_batch=8, tol=1e-10)
    m = srv.add_model(A, part, p, rank_k=6, **MC)
    b = W.rhs(A[0], 9)
    x_alone, inf_alone, _, _ = srv.wait(srv.submit(m, b), A[0])
    r0 = srv.submit(m, b)
    more = [srv.submit(m, W.rhs(A[0], 50 + i)) for i in range(7)]
    x0, inf0, _, bw0 = srv.wait(r0, A[0])
    outs = [srv.wait(r, A[0]) for r in more]
    assert np.array_equal(x0, x_alone) and inf0["its"] == inf_alone["its"]
    assert all(o[1]["status"] == "OK" and o[1]["relres"] <= 1e-10 for o in outs)
    assert max(o[3] for o in outs) > 1
    srv.close()


def test_narrowing_keeps_running_columns():
    """Zero right-hand sides finish at admission; the block is then narrowed
    to the one running column, whose result is still bitwise its result
    alone (a zero right-hand side gives x = 0 in no iteration)."""
    A, part, p = _problem((20, 20, 20), (2, 2, 2))
    srv = pkg.Server(max_concurrent=1, max_batch=8, tol=1e-10)
    m = srv.add_model(A, part, p, rank_k=6, **MC)
    b = W.rhs(A[0], 11)
    x_alone, inf_alone, _, bw_alone = srv.wait(srv.submit(m, b), A[0])
    ids = [srv.submit(m, np.zeros(A[0])) for _ in range(3)]
    r = srv.submit(m, b)
    ids += [srv.submit(m, np.zeros(A[0])) for _ in range(4)]
    zs = [srv.wait(i, A[0]) for i in ids]
    x, inf, _, bw = srv.wait(r, A[0])
    assert all(z[1]["its"] == 0 and not np.any(z[0]) for z in zs)
    assert np.array_equal(x, x_alone) and inf["its"] == inf_alone["its"]
    srv.close()


def test_poisson_stream_small():
    from paper_1505_04341_gb300 import serve
    srv, models = serve.setup_server([32, 48], k=8, max_batch=8)
    recs, mk = serve.run_stream(srv, models, nreq=24, rate=200.0)
    s = serve.summarize(recs, mk)
    assert s["all_ok"] and s["max_relres"] <= 1e-8 and s["requests"] == 24
    assert s["latency_p99_ms"] >= s["latency_p50_ms"] > 0
    srv.close()
