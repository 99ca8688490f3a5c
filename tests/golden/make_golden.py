"""Write the stored oracle results for the full-size benchmark instances.

Calls only the CPU oracle (oracle/) on inputs from the seeded generators and
writes tests/golden/<workload>.json with the input digest, the oracle's radius,
centre, active set and KKT residuals.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2605_31425_gb300 import workloads  # noqa: E402


def main(names):
    for name in names:
        C, R = workloads.workload(name)
        t = time.time()
        res = oracle.solve(C, R, tol=1e-12)
        dt = time.time() - t
        out = dict(
            workload=name, m=int(C.shape[0]), d=int(C.shape[1]),
            input_sha256=workloads.digest(C, R),
            r=res["r"], r_alm=res["r_alm"], c=[float(v) for v in res["c"]],
            active=[int(i) for i in res["active"]], kkt_max=res["kkt_max"],
            status=res["status"], outer_iters=res["outer_iters"], ssn_iters=res["ssn_iters"],
            passes=res["passes"], oracle_seconds=dt, tol=1e-12,
            note="written by tests/golden/make_golden.py from oracle.solve; inputs from "
                 "paper_2605_31425_gb300.workloads.workload(name)",
        )
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, res["r"], res["status"], f"{dt:.1f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["cube_m2e6_d100", "gaussian_m1e4_d10"])
