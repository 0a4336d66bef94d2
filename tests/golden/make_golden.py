"""Write tests/golden/c1_samples.json from the oracle alone.

Workload: unit Gaussian, sigma = 0.15, at the centre of [-1,1]^3 on 32^3 cells
(the paper's Sec. 3 three-dimensional test, on the doubled box).  Stores the
FP64 oracle's phi and E for HE and VGF at 24 seeded cells, with the closed-form
values beside them.  The paper prints no numbers; these values come from the
committed oracle and the erf closed form only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from oracle import analytic as A  # noqa: E402


def main():
    prob = W.unit_gaussian_3d(32, 0.15, 2.0)
    rho = prob.rho(np.float32).astype(np.float64)
    rng = np.random.default_rng(2024)
    cells = rng.integers(0, 32, size=(24, 3))
    idx = tuple(cells.T)
    pts = W.grid_points(prob.shape, prob.h)[idx]
    pex, Eex = A.mixture_field(pts, prob.gaussians, 3)
    out = {"workload": "unit Gaussian sigma=0.15 at origin, [-1,1]^3, 32^3 cells, rho rounded to FP32",
           "cells": cells.tolist(), "closed_form": {"phi": pex.tolist(), "E": Eex.T.tolist()}}
    for method in ("he", "vgf"):
        phi, E = oracle.solve(method, rho, prob.h)
        out[method] = {"phi": phi[idx].tolist(), "E": E[(slice(None),) + idx].T.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_samples.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
