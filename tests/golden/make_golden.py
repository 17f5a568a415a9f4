"""Write tests/golden/c1_oracle.json: oracle-only reference values for the 64x32 O-mesh, 16x16
velocity-grid, Kn=1, Ma=0.5 workload (drag, Cd, both sensitivities over the 8 bump amplitudes).

Calls only oracle/ and the seeded input generators.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                      # noqa: E402
from paper_2501_00923_gb300 import workloads as W   # noqa: E402


def main():
    wl = W.config(0)
    pr = O.Problem.from_workload(wl)
    t = time.time()
    f, info = pr.primal_solve(tol=1e-13, max_sweeps=40000)
    phi, ainfo = pr.adjoint_solve(f, tol=1e-13, max_sweeps=40000)
    J = pr.functional(f)
    U = wl.flow.Ma * W.A_INF
    g_full = pr.sens_full(f, phi, wl.mesh.dnodes())
    g_paper, node_paper, _ = pr.sens_paper(f, phi, wl.mesh.dwall)
    lift = O.Problem.from_workload(wl, direction=(0.0, 1.0)).functional(f)
    out = {
        "workload": wl.name,
        "source": "oracle/dvm_oracle.cpp via tests/golden/make_golden.py",
        "primal": info, "adjoint": ainfo,
        "J": J, "Cd": J / (0.5 * U * U), "lift": lift,
        "grad_full": g_full.tolist(), "grad_paper": g_paper.tolist(),
        "seconds": time.time() - t,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
