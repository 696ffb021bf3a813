"""Work counts of the oracle's own time steps on a benchmark workload, stored
for the CPU reference timing: MLSDC iterations, multigrid V-cycles and
V-cycle work (sum over V-cycles of the solved grid's N^3) per step.

TEST INFRASTRUCTURE ONLY (it runs the oracle, nothing else).  The reference
timing in bench.py times one fine V-cycle and one iteration's remaining work
on the host cores and scales them by these counts, because a full oracle time
step at 255^3 takes tens of minutes.

    python oracle/step_counts.py [workload ...]   (default: c2)

runs the OpenMP build of the oracle for the first two steps of each workload
at its full size and writes oracle/step_counts.json.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
# run as a script, this folder would shadow the package of the same name
sys.path[:] = [ROOT] + [p for p in sys.path if os.path.abspath(p or ".") != HERE]

OUT = os.path.join(HERE, "step_counts.json")
STEPS = 2


def counts(name: str) -> dict:
    from bench import WORKLOADS
    from oracle import oracle as O
    from paper_1307_7867_gb300 import inputs
    w = WORKLOADS[name]
    if w["slices"] != 1 or w["precision"] != "fp64":
        raise SystemExit(f"{name}: only serial FP64 workloads are counted")
    prob = O.Prob(nu=0.1, forcing=1, kappa=1.0, mg_tol=w["mg_tol"], mg_max=50,
                  interp=w.get("interp", 2))
    u0 = inputs.sine_mode(w["fine"][0])
    t0 = time.time()
    with O.openmp():
        if w["coarse"]:
            uT, rc, st = O.mlsdc_run(w["fine"], w["coarse"], prob, w["dt"], STEPS, u0,
                                     nsweeps_fine=w["sweeps_fine"],
                                     nsweeps_coarse=w["sweeps_coarse"], max_iters=w["iters"],
                                     tol=w["tol_sdc"])
        else:
            uT, rc, st = O.sdc_run(*w["fine"], prob, w["dt"], STEPS, w["sweeps_fine"], u0,
                                   tol=w["tol_sdc"])
    # an iteration of a single-level workload is one SDC sweep
    its = st["iters"] if w["coarse"] else st["sweeps"]
    return {"workload": w["desc"], "steps": STEPS, "status": rc,
            "iters_per_step": its / STEPS, "vcycles_per_step": st["vcycles"] / STEPS,
            "solves_per_step": st["solves"] / STEPS,
            "vcycle_points_per_step": st["vcycle_points"] / STEPS,
            "oracle_seconds": round(time.time() - t0, 1), "threads": os.cpu_count()}


def main():
    names = sys.argv[1:] or ["c2"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in names:
        data[n] = counts(n)
        print(n, data[n], flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
