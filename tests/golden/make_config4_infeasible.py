"""Write config4_infeasible_full.json: the oracle's step on the full-size infeasible
centre-of-mass workload (3D 256x128x128, n = 4,194,304, four coupled rows, the target
outside the domain), whose exact coupled solve takes minutes of CPU time.

Only the oracle and the seeded input generator are called.  The test that reads the
file recomputes the step from the seed with these multipliers given
(oracle_step(..., lam_given=...)) and checks them against the KKT conditions of that
problem before it compares the device result with them.

    python tests/golden/make_config4_infeasible.py
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.step import oracle_step  # noqa: E402
from paper_2511_13905_gb300 import inputs  # noqa: E402


def main():
    cfg = inputs.config4(infeasible=True)
    t0 = time.time()
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"],
                      cfg["G"], cfg["t"], mode="coupled")
    out = {
        "source": "oracle.step.oracle_step (exact coupled projector) on inputs.config4(infeasible=True), "
                  "written by tests/golden/make_config4_infeasible.py",
        "workload": cfg["name"], "n": cfg["n"], "m": cfg["m"],
        "lam": [float(v) for v in ref["lam"]], "b": [float(v) for v in ref["b"]],
        "alpha": ref["alpha"], "beta": ref["beta"], "branch": ref["branch"],
        "rel_change": ref["rel_change"],
        "row_sets_tried": ref["info"]["row_sets_tried"], "kkt_worst": ref["info"]["kkt"]["worst"],
        "cpu_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, "config4_infeasible_full.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
