"""Record the oracle's own FGMRES iteration count on the bench workload.

TEST INFRASTRUCTURE ONLY.  Runs the complex128 oracle (sweeping-preconditioned
FGMRES, Sections 4-6 of the paper) to a relative residual of 1e-6 on the
1023 x 1023, 8 x 8 workload and writes oracle/reference_counts.json.  The CPU
baseline of bench.py times a bounded sample of oracle iterations and scales it
by this count.  Calls only oracle/ and workloads/ (minutes to an hour of CPU).

    python oracle/reference_counts.py BSP 200
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import Decomposition, Sweeper, assemble_operator, fgmres  # noqa: E402


def main(sched="BSP", restart=200, workload="plain_mixed"):
    w = W.workload(workload)
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    sw = Sweeper(dec)
    t0 = time.perf_counter()
    hist = []
    x, it, rr = fgmres(lambda v: A @ v, lambda v: sw.precondition(v, sched), w.h ** 2 * w.f[0], tol=1e-6,
                       restart=restart, maxit=5000, history=hist)
    dt = time.perf_counter() - t0
    path = os.path.join(ROOT, "oracle", "reference_counts.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    d.setdefault(workload, {})[f"{sched}_restart{restart}"] = {
        "iterations": it, "relres": rr, "seconds": dt, "transmission": "optimized, scale 1.0", "tol": 1e-6}
    json.dump(d, open(path, "w"), indent=1, sort_keys=True)
    print(it, rr, dt)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "BSP", int(sys.argv[2]) if len(sys.argv) > 2 else 200)
