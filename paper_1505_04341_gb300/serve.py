"""Serving driver: a stream of solve requests over several grid sizes.

Each request is a 3-D 7-point Laplacian solve with the grid edge drawn
uniformly from a set of edges, (edge/16)^3 box subdomains, one random
right-hand side, arriving as a Poisson process.  The models (one per edge) are
set up once and stay resident in the server; requests are submitted at their
arrival times and the driver records the latency of each (submit to result) and
the throughput.

    python -m paper_1505_04341_gb300.serve --requests 512 --rate 0   # saturated
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def setup_server(edges, k=16, max_batch=16, max_concurrent=8, tol=1e-8):
    import workloads as W
    from paper_1505_04341_gb300 import Server
    srv = Server(max_concurrent=max_concurrent, max_batch=max_batch, tol=tol)
    models = {}
    for e in edges:
        w = W.workload(f"lap3d_{e}")
        t0 = time.perf_counter()
        models[e] = (srv.add_model(w["A"], w["part"], w["p"], variant=1, rank_k=k, c_order=1,
                                   b_order=1), w["A"][0], time.perf_counter() - t0)
    return srv, models


def run_stream(srv, models, nreq=512, rate=0.0, seed=0):
    """Submits nreq requests (edge uniform over the models, RHS from SplitMix64
    stream seed+i) with Poisson arrivals at `rate` per second (0: all at once);
    returns per-request records and the makespan."""
    import workloads as W
    edges = sorted(models)
    u = W.uniform01(seed, 2 * nreq)
    pick = [edges[min(len(edges) - 1, int(u[2 * i] * len(edges)))] for i in range(nreq)]
    gaps = (-np.log1p(-u[1::2]) / rate) if rate > 0 else np.zeros(nreq)
    arrivals = np.cumsum(gaps)
    rhs = [W.rhs(models[e][1], 1000 + i) for i, e in enumerate(pick)]
    ids = [None] * nreq
    t0 = time.perf_counter()

    def submitter():
        for i in range(nreq):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids[i] = srv.submit(models[pick[i]][0], rhs[i])

    th = threading.Thread(target=submitter)
    th.start()
    recs = []
    for i in range(nreq):
        while ids[i] is None:
            time.sleep(1e-4)
        x, info, lat, bw = srv.wait(ids[i], models[pick[i]][1])
        recs.append(dict(edge=pick[i], its=info["its"], relres=info["relres"],
                         status=info["status"], latency=lat, batch=bw))
    th.join()
    return recs, time.perf_counter() - t0


def summarize(recs, makespan):
    lat = np.array([r["latency"] for r in recs])
    return {"requests": len(recs), "solves_per_s": round(len(recs) / makespan, 2),
            "makespan_s": round(makespan, 3),
            "latency_p50_ms": round(1e3 * float(np.percentile(lat, 50)), 2),
            "latency_p99_ms": round(1e3 * float(np.percentile(lat, 99)), 2),
            "all_ok": all(r["status"] == "OK" for r in recs),
            "max_relres": max(r["relres"] for r in recs),
            "mean_batch": round(float(np.mean([r["batch"] for r in recs])), 2)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--edges", default="32,48,64,96,128")
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals per second (0: saturate)")
    ap.add_argument("--loads", default="", help="comma list of fractions of the saturated rate")
    args = ap.parse_args(argv)
    edges = [int(e) for e in args.edges.split(",")]
    srv, models = setup_server(edges)
    out = {"edges": edges, "setup_s": {str(e): round(models[e][2], 3) for e in edges}}
    recs, mk = run_stream(srv, models, args.requests, args.rate)
    out["run"] = summarize(recs, mk)
    if args.loads:
        sat = out["run"]["solves_per_s"]
        for f in [float(v) for v in args.loads.split(",")]:
            r2, mk2 = run_stream(srv, models, args.requests, f * sat, seed=1)
            out[f"load_{f}"] = summarize(r2, mk2)
    out["stats"] = srv.stats()
    srv.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
