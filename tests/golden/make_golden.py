"""Writes the stored expected values under tests/golden/ from the oracle.

The paper prints no worked numeric example for the trajectory-optimisation
path (its tables are timings), so these fixtures are regression records of
the pinned FP64 oracle on small seeded problems: a later change to the
oracle's arithmetic shows up as a mismatch and must say which passage
justifies it.  Only the oracle and the seeded generator are called.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2602_19699_gb300 import workload as W  # noqa: E402

CASES = {
    # system, seed, batch seed, B, T, max_iter
    "pointmass_T10": (W.POINTMASS, 1, 2, 3, 10, 6),
    "planar3_T12": (W.PLANAR3, 1, 2, 2, 12, 4),
    "dubins_T12": (W.DUBINS, 1, 2, 2, 12, 5),
}


def compute(name):
    sysid, seed, bseed, B, T, iters = CASES[name]
    prob = W.make_problem(sysid, seed)
    b = W.make_batch(prob, B, seed=bseed, T=T)
    r = oracle.Oracle.from_problem(prob).solve(b.x0, b.T, max_iter=iters, tol=1e-8, n_alpha=16)
    return {"system": int(sysid), "seed": seed, "batch_seed": bseed, "B": B, "T": T, "max_iter": iters,
            "x0": b.x0.tolist(), "J": r["J"].tolist(), "iters": r["iters"].tolist(), "status": r["status"].tolist(),
            "alpha_hist": r["alpha_hist"].tolist(), "U": r["U"].tolist(), "X_T": r["X"][:, -1].tolist()}


if __name__ == "__main__":
    for name in CASES:
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(compute(name), f, indent=1)
        print("wrote", name)
