"""GPU: the solve service (continuous batching across requests and models).
A request's result is the same alone and in a mix of concurrent requests (the
batched solve gives a column the same bits whatever shares its batch), and
every result meets the tolerance and agrees with a direct solve."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def test_alone_equals_in_the_mix():
    srv = pkg.Server(max_concurrent=3, max_batch=8, tol=1e-8)
    probs = {}
    for shape, parts in (((16, 16, 16), (2, 2, 2)), ((24, 20, 18), (3, 2, 2))):
        A = W.laplacian(shape)
        part, p = W.box_partition(shape, parts)
        probs[shape] = (srv.add_model(A, part, p, rank_k=8, c_order=1, b_order=1), A)
    (m0, A0), (m1, A1) = probs[(16, 16, 16)], probs[(24, 20, 18)]
    b0 = W.rhs(A0[0], 5)
    x_alone, inf, _, bw = srv.wait(srv.submit(m0, b0), A0[0])
    assert inf["status"] == "OK" and inf["relres"] <= 1e-8 and bw == 1
    # the same request inside a burst of requests on both models
    ids = []
    for i in range(12):
        ids.append((m1, A1[0], srv.submit(m1, W.rhs(A1[0], 100 + i))))
        ids.append((m0, A0[0], srv.submit(m0, W.rhs(A0[0], 200 + i))))
        if i == 5:
            ids.append((m0, A0[0], srv.submit(m0, b0)))
            mark = len(ids) - 1
    res = [srv.wait(r, n) for (_, n, r) in ids]
    x_mix, inf_mix, _, bw_mix = res[mark]
    assert inf_mix["status"] == "OK"
    assert np.array_equal(x_alone, x_mix)                 # same bits
    assert all(r[1]["status"] == "OK" and r[1]["relres"] <= 1e-8 for r in res)
    st = srv.stats()
    assert st["max_batch_seen"] > 1                       # requests were batched
    # agreement with a direct solve on a plain handle
    h = pkg.DDLR(A0, *W.box_partition((16, 16, 16), (2, 2, 2)), rank_k=8, c_order=1, b_order=1)
    xd, infd = h.pcg(b0, tol=1e-8)
    assert np.abs(xd - x_alone).max() / np.abs(xd).max() < 1e-6
    h.close()
    srv.close()


def test_poisson_stream_small():
    from paper_1505_04341_gb300 import serve
    srv, models = serve.setup_server([32, 48], k=8, max_batch=8)
    recs, mk = serve.run_stream(srv, models, nreq=24, rate=200.0)
    s = serve.summarize(recs, mk)
    assert s["all_ok"] and s["max_relres"] <= 1e-8 and s["requests"] == 24
    assert s["latency_p99_ms"] >= s["latency_p50_ms"] > 0
    srv.close()
