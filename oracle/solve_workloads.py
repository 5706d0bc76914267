"""Run the oracle's FP64 CG to convergence on a named workload and store its
iteration count and true residual in ``oracle/workload_solves.json``.

TEST INFRASTRUCTURE: calls only ``oracle`` and ``fieldgen``.  The stored
iteration count lets a bounded timing sample of the oracle (a few CG
iterations) be scaled to the time of a full solve.

    python -m oracle.solve_workloads cfg32
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import fieldgen as fg  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "workload_solves.json")


def solve(name: str, tol: float = 1e-10, maxiter: int = 200000) -> dict:
    wl = fg.workload(name)
    u, w, b = fg.make_inputs(wl["dims"], wl["fat"], wl["naik"], wl["seed"], wl["a"])
    c3 = -1.0 / 24.0 if wl["naik"] else 0.0
    t0 = time.time()
    x, ok, iters, tr = oracle.cg(wl["dims"], u, b, wl["mass"], w, c3, tol=tol, maxiter=maxiter)
    return {"workload": name, "dims": list(wl["dims"]), "mass": wl["mass"], "tol": tol, "converged": bool(ok),
            "iters": iters, "true_rel_resid": tr, "seconds": round(time.time() - t0, 1),
            "threads": oracle.threads()}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        data[n] = solve(n)
        print(json.dumps(data[n]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["cfg4x4", "cfg32"])
