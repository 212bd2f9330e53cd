"""Small, fixed solves for profiling one solver launch under ncu.

    python -m paper_2602_19699_gb300.profile_cases planar3 mixed 8192 3
    python -m paper_2602_19699_gb300.profile_cases quad mixed 608 1 10

planar3: the benchmark's planar-arm workload (seed 0, T ~ U{100..400}) cut to
B instances and max_iter iterations; quad: B quadruped instances of horizon
T with the zero-control warm start.  Each runs one solve (one solver
launch) and prints the mean iteration count.
"""
from __future__ import annotations

import sys


def main(argv):
    from . import Solver, TO_FP64, TO_MIXED, build
    from . import workload as W
    system = argv[0] if argv else "planar3"
    prec = TO_MIXED if (len(argv) < 2 or argv[1] == "mixed") else TO_FP64
    B = int(argv[2]) if len(argv) > 2 else 1024
    max_iter = int(argv[3]) if len(argv) > 3 else 3
    build()
    if system == "planar3":
        prob = W.planar3(seed=0)
        b = W.make_batch(prob, B, seed=0)
        T_max = 400
    elif system == "quad":
        T = int(argv[4]) if len(argv) > 4 else 10
        prob = W.quad(seed=0, with_actor=False)
        b = W.make_batch(prob, B, seed=0, T=T)
        T_max = T
    else:
        raise SystemExit(f"unknown case {system!r}")
    r = Solver(prob, T_max=T_max, prec=prec).solve(b.x0, b.T, max_iter=max_iter, history=False)
    print("ok", float(r["iters"].mean()))


if __name__ == "__main__":
    main(sys.argv[1:])
