"""Write the stored expected values of tests/golden/ from the FP64 oracle.

The paper prints no worked example with solution values (Section 3 reports
timings and the iterative solver's mean differences on an unavailable MONC case),
so the fixtures here come from the oracle only: the zero-mean solution of L p = Q_W S
(Section 2.1), p = L^-1 S with p = 0 on the top face, and the variable-density
solve of the conjugate-gradient path (Section 2.2's iterative route), on tiny
seeded grids.  Each case stores its inputs' recipe, every solution value and
two norms, so the tests can re-derive the inputs and compare element by element.

    python tests/golden/make_golden.py      # rewrites oracle_small_cases.json
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2010_14132_gb300 import workloads as wl  # noqa: E402

CASES = [
    {"name": "uniform_8x8x8_neumann", "kind": "uniform", "n": 8, "seed": 11, "bc": "neumann"},
    {"name": "stretched_6x4x5_neumann", "kind": "stretched", "dims": [6, 4, 5], "seed": 12, "bc": "neumann"},
    {"name": "stretched_8x6x5_dirichlet_top", "kind": "stretched", "dims": [8, 6, 5], "seed": 13,
     "bc": "dirichlet_top"},
    {"name": "variable_density_6x4x4_neumann", "kind": "variable", "dims": [6, 4, 4], "seed": 14, "eps": 0.3,
     "bc": "neumann"},
]


def inputs(case):
    """The case's domain (and density field) from the seeded generators."""
    if case["kind"] == "uniform":
        d = wl.uniform_cube(case["n"], seed=case["seed"])
        return d, None
    d = wl.random_stretched(*case["dims"], seed=case["seed"])
    rho3 = None
    if case["kind"] == "variable":
        rho3 = wl.perturbed_density(d.nx, d.ny, d.rho0, case["eps"], seed=case["seed"] + 1)
    return d, rho3


def solve(case):
    d, rho3 = inputs(case)
    if rho3 is not None:
        return O.solve_var(d.S, d.dx, d.dy, d.dz, rho3, case["bc"])
    return O.solve(d.S, d.dx, d.dy, d.dz, d.rho0, bc=case["bc"])


def main():
    out = {"_source": "FP64 oracle (oracle/poisson_oracle.py) on the seeded inputs described per case",
           "cases": []}
    for case in CASES:
        p = solve(case)
        out["cases"].append(dict(case, shape=list(p.shape), l2=float(np.linalg.norm(p)),
                                 mean=float(p.mean()), p=[float(v) for v in p.ravel()]))
    with open(os.path.join(HERE, "oracle_small_cases.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
