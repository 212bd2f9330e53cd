"""Writes tests/golden/quad_oracle_B8_T100.json: the FP64 oracle's solve of
the first 8 instances of the quadruped workload (seed 0 problem with its
actor warm start, batch seed 0, T = 100), 20 iterations, 16 step sizes.

The oracle takes about 5 s per iteration and instance on one host core for
this system (48 tangent directions through 10 contact substeps per knot), so
the benchmark cannot solve it while it runs; it reads this record instead
and compares the GPU's solve of the same instances with it.  A second solve
with x0 moved by 1e-15 relative records the oracle's own reproducibility.
Only the oracle and the seeded generator are called.

    python tests/golden/make_quad_reference.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2602_19699_gb300 import workload as W  # noqa: E402

B_SAMPLE, B_FULL, T, MAX_ITER, N_ALPHA, KNOT_STRIDE = 8, 2048, 100, 20, 16, 10


def compute():
    prob = W.quad(seed=0)
    b = W.make_batch(prob, B_FULL, seed=0, T=T)
    x0, Ts = b.x0[:B_SAMPLE], b.T[:B_SAMPLE]
    o = oracle.Oracle.from_problem(prob)
    threads = os.cpu_count() or 1
    r = o.solve(x0, Ts, max_iter=MAX_ITER, tol=1e-8, n_alpha=N_ALPHA, threads=threads)
    x1 = x0 * (1 + 1e-15 * np.random.default_rng(1).choice([-1.0, 1.0], size=x0.shape))
    r1 = o.solve(x1, Ts, max_iter=MAX_ITER, tol=1e-8, n_alpha=N_ALPHA, threads=threads)
    knots = list(range(0, T + 1, KNOT_STRIDE))
    return {"system": int(W.QUAD), "problem_seed": 0, "batch_seed": 0, "B_full": B_FULL, "sample": B_SAMPLE,
            "T": T, "max_iter": MAX_ITER, "n_alpha": N_ALPHA, "tol": 1e-8, "warm_start": "actor",
            "x0": x0.tolist(), "J": r["J"].tolist(), "status": r["status"].tolist(), "iters": r["iters"].tolist(),
            "alpha_hist": r["alpha_hist"].tolist(), "J_hist": r["J_hist"].tolist(), "knots": knots,
            "X_knots": r["X"][:, knots].tolist(),
            "perturbed_x0_1e-15": {"J": r1["J"].tolist(), "X_knots": r1["X"][:, knots].tolist()}}


if __name__ == "__main__":
    out = compute()
    with open(os.path.join(HERE, "quad_oracle_B8_T100.json"), "w") as f:
        json.dump(out, f)
    print("wrote quad_oracle_B8_T100.json")
