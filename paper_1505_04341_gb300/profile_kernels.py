"""Kernel driver for profiling and timing one operation of the library.

Builds the preconditioner for a named workload and repeats one operation --
an A0 solve, an M^-1 apply, a PCG solve, a GMRES(40) solve (`gmres`, with
--indefinite 1 for a preconditioner that is not SPD, --factor and
--fill-level for the local factors) or the device setup from resident values
(factorisation and Lanczos, `setup`) -- with device-resident vectors,
printing the CUDA-event time per repetition and the algorithmic bytes.  Used
as the command under ncu for the kernel summaries in profiles/:

    python -m paper_1505_04341_gb300.profile_kernels --workload lap3d_128_b8 \
        --op a0 --reps 5 [--variant 1] [--k 16] [--precision 0] [--c-solver 0]
        [--families]

--families adds a second pass with per-launch CUDA events (ddlr_set_timing)
and prints the device time, launches and algorithmic GB/s of every kernel
family.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lap3d_64_b4")
    ap.add_argument("--op", default="a0", choices=["a0", "apply", "pcg", "setup", "gmres"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--variant", type=int, default=1)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--bf16", type=int, default=1)
    ap.add_argument("--c-order", type=int, default=1)
    ap.add_argument("--b-order", type=int, default=1)
    ap.add_argument("--lanczos-max", type=int, default=0)
    ap.add_argument("--c-solver", type=int, default=0)
    ap.add_argument("--families", action="store_true")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--scale-diag", type=int, default=0)
    ap.add_argument("--maxit", type=int, default=500)
    ap.add_argument("--factor", type=int, default=0)
    ap.add_argument("--fill-level", type=int, default=0)
    ap.add_argument("--indefinite", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-8)
    args = ap.parse_args(argv)

    import torch

    import workloads as W
    from paper_1505_04341_gb300 import DDLR, DdlrError, build

    build()
    w = W.workload(args.workload)
    A, part, p = w["A"], w["part"], w["p"]
    n = A[0]
    h = DDLR(A, part, p, variant=args.variant, rank_k=args.k, factor=args.factor, fill_level=args.fill_level,
             indefinite=args.indefinite,
             c_order=args.c_order, b_order=args.b_order, precision=args.precision,
             uk_bf16=args.bf16, c_solver=args.c_solver, scale_diag=args.scale_diag,
             max_nrhs=args.nrhs, lanczos_max=args.lanczos_max)
    if args.nrhs == 1:
        b = torch.tensor(W.rhs(n, 0), device="cuda")
    else:   # n x nrhs column-major block
        import numpy as np
        b = torch.tensor(np.stack([W.rhs(n, s) for s in range(args.nrhs)], axis=1), device="cuda").T.contiguous().T
    y = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    def once():
        if args.op == "a0":
            h.a0_solve(b, y)
        elif args.op == "apply":
            h.apply(b, y)
        elif args.op == "setup":
            h.refactor()
        elif args.op == "gmres":    # GMRES(40); a capped step count profiles the same kernels
            h.gmres(b, y, tol=args.tol, maxit=args.maxit, check=False)
        else:
            try:
                h.pcg(b, y, tol=1e-8, maxit=args.maxit)
            except DdlrError as e:      # a capped iteration count profiles the same kernels
                if e.status != "NOCONV":
                    raise

    once()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        once()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    tr = h.traffic()
    byts = tr["a0_bytes"] if args.op == "a0" else tr["apply_bytes"]
    best = min(times)
    fam = None
    if args.families:
        h.reset_counters()
        h.set_timing(True)
        for _ in range(args.reps):
            once()
        torch.cuda.synchronize()
        h.set_timing(False)
        cnt = h.counters()["families"]
        fb = h.traffic()["family_bytes"]
        fam = {f: {"us_per_launch": round(v["ms"] * 1e3 / v["launches"], 2),
                   "launches_per_rep": v["launches"] / args.reps,
                   "GBps": (round(fb.get(f, 0) / (v["ms"] * 1e-3 / v["launches"]) / 1e9, 1)
                            if fb.get(f, 0) > 0 and v["ms"] > 0 else None)}
               for f, v in cnt.items() if v["launches"] > 0}
    print(json.dumps({"workload": args.workload, "op": args.op, "ms": times, "families": fam,
                      "best_ms": best, "algorithmic_bytes": byts,
                      "GBps_best": byts / (best * 1e-3) / 1e9 if args.op in ("a0", "apply") else None,
                      "info": {k: v for k, v in h.info().items()
                               if k in ("n", "s", "p", "k", "levels_interior", "levels_c",
                                        "nnz_factor", "lanczos_steps")}}))
    h.close()


if __name__ == "__main__":
    main()
