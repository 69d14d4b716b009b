"""Writes oracle_regression.json: the oracle's PCG solves of three small seeded
problems (iterations, final relative residual, solution norm and a few
entries), to catch unintended changes of the oracle's arithmetic.  Calls only
oracle/ and the input generators; run from the repository root:

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import discretize, mg  # noqa: E402
from paper_1902_01818_gb300 import workloads as W  # noqa: E402

CASES = {
    "conf2d_unit_square_n8_p2_scms": (lambda: W.unit_square_2x2(n=8, p=2)[0], 2, "scms", 1.0, 0.12),
    "sipg2d_3x3_n4_8_p3_hybrid": (lambda: W.grid_problem((3, 3), lambda c, a: 4 if sum(c) % 2 == 0 else 8, 3,
                                                         "sipg", jitter=0.1, seed=2), 2, "hybrid", 0.25, 0.1),
    "conf3d_2x2x2_n4_p2_hybrid": (lambda: W.grid_problem((2, 2, 2), 4, 2, "conforming", jitter=0.05, seed=3,
                                                         jitter_boundary_tangential=True), 2, "hybrid", 0.25, 0.12),
}


def solve_case(name):
    fac, levels, smoother, tau, delta = CASES[name]
    prob = fac()
    M = mg.Multigrid(prob, levels=levels, smoother=smoother, tau=tau, delta=delta)
    f = discretize.assemble_load(prob, prob["knots"], M.h["num"][-1], W.source_sinprod)
    u, it, hist = M.solve_pcg(f, tol=1e-8)
    return {"ndof": int(M.ndof), "iterations": int(it), "final_relres": float(hist[-1]),
            "u_norm": float(np.linalg.norm(u)), "u_head": [float(x) for x in u[:4]]}


if __name__ == "__main__":
    out = {name: solve_case(name) for name in CASES}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))
