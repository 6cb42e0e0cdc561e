"""Writes oracle_solves.json: the CPU oracle's own whole solves of the named
workloads (the exact-Cholesky FP64 IPM of Algorithm 3 from the infeasible
start x0 = s0 = 1, y0 = 0, tolerance 1e-8), one record per workload: outer
iterations, objective, final relative gap and residuals, and the wall time on
the machine that ran it.  Calls only lpgen (the inputs) and oracle/.

The bench's CPU baseline for a workload too large to solve whole within its
run times single outer iterations of the oracle live and scales them by the
outer-iteration count recorded here for the same LP; the bench also checks the
GPU objective against the objective recorded here.

    python tests/golden/make_oracle_records.py c4 [c2 c3 ...]
"""

import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lpgen  # noqa: E402
from oracle import ipm  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solves.json")


def record(name: str) -> dict:
    cfg = lpgen.CONFIGS[name]
    lp = lpgen.make(cfg)
    if lp.sparse:  # the oracle's exact solver takes the sparse matrix as it is
        import scipy.sparse as sps
        A = sps.csc_matrix((lp.val, lp.row_idx, lp.col_ptr), shape=(lp.m, lp.n))
    else:
        A = lp.dense()
    t0 = time.perf_counter()
    res = ipm.solve(A, lp.b, lp.c, ipm.Options(mode="infeasible", solver="exact", tol=1e-8))
    secs = time.perf_counter() - t0
    last = res.history[-1]
    cx = float(lp.c @ res.x)
    return {
        "workload": name, "m": lp.m, "n": lp.n, "storage": lp.storage, "seed": cfg["seed"],
        "status": res.status, "outer_iterations": res.iterations,
        "objective": cx, "planted_objective": lp.objective,
        "objective_rel_err_vs_planted": abs(cx - lp.objective) / (1 + abs(lp.objective)),
        "rel_gap": last.gap,
        "rp_rel": last.rp_norm / (1 + float(np.linalg.norm(lp.b))),
        "rd_rel": last.rd_norm / (1 + float(np.linalg.norm(lp.c))),
        "seconds": secs, "seconds_per_outer_iteration": secs / max(1, res.iterations),
        "cores": os.cpu_count(), "machine": platform.machine(),
    }


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = record(name)
        print(json.dumps(data[name]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["c4"])
