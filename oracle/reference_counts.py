"""Record the oracle's own iteration counts on the bench workload.

TEST INFRASTRUCTURE ONLY.  Runs the complex128 oracle to a relative residual of
1e-6 on the 1023 x 1023, 8 x 8 workload and writes oracle/reference_counts.json;
the CPU baseline of bench.py times a bounded sample of the oracle and scales it
by these counts.  Calls only oracle/ and workloads/.

Two methods:
* ``single``: volume FGMRES(restart) preconditioned by one sweep per application
  (Robin scale 1.0);
* ``interface``: the bench's default method, the paper's formulation: volume
  FGMRES(restart) whose preconditioner solves the interface problem
  (I - S) g = b by FGMRES(30) to 1e-2 (at most 300 steps) with the sweep as its
  preconditioner (Sections 3-5), Robin scale 0.5; records the outer steps and
  the interface steps summed over the preconditioner applications.

    python oracle/reference_counts.py single BSP 150
    python oracle/reference_counts.py interface BSP 150
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import Decomposition, Sweeper, assemble_operator, fgmres  # noqa: E402

INNER = dict(tol=1e-2, restart=30, maxit=300)     # the interface iteration of the bench's default method


def main(method="interface", sched="BSP", restart=150, workload="plain_mixed"):
    w = W.workload(workload)
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    scale = 0.5 if method == "interface" else 1.0
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, tc_scale=scale)
    sw = Sweeper(dec)
    if method == "interface":
        pre = lambda v: sw.precondition_interface_krylov(v, sched, **INNER)
    else:
        pre = lambda v: sw.precondition(v, sched)
    t0 = time.perf_counter()
    hist = []
    x, it, rr = fgmres(lambda v: A @ v, pre, w.h ** 2 * w.f[0], tol=1e-6, restart=restart, maxit=5000, history=hist)
    dt = time.perf_counter() - t0
    path = os.path.join(ROOT, "oracle", "reference_counts.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    key = f"{sched}_restart{restart}" if method == "single" else f"{sched}_interface_krylov_restart{restart}"
    entry = {"iterations": it, "relres": rr, "seconds": dt, "transmission": f"optimized, scale {scale:g}", "tol": 1e-6}
    if method == "interface":
        entry.update(interface_steps=sw.interface_steps, inner=INNER)
    d.setdefault(workload, {})[key] = entry
    json.dump(d, open(path, "w"), indent=1, sort_keys=True)
    print(key, entry)


if __name__ == "__main__":
    a = sys.argv[1:]
    main(a[0] if a else "interface", a[1] if len(a) > 1 else "BSP", int(a[2]) if len(a) > 2 else 150)
