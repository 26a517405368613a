"""Command-line solve of one control problem (beta^2 A^-alpha + gamma A^alpha) u = beta y_Omega
with a seeded synthetic right-hand side:

    python -m paper_1809_01971_gb300 --problem 5 --precision 2 --repeats 3

--problem k selects the k-th 3D n = 255 problem (alpha in {0.25, 0.5, 0.75} x gamma in
{1e-1, 1e-3}: four separable Gaussians + one grid sine mode), --problem 2d the 2D n = 63 one.
--precision picks the contraction form (0 FP64, 1 double-float FP32, 2 tensor-core digit
products).  Prints the PCG summary and the device time of each solve (CUDA events).
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    p = argparse.ArgumentParser(prog="python -m paper_1809_01971_gb300")
    p.add_argument("--problem", default="5", help="0..5 (3D, n=255) or 2d (n=63)")
    p.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    p.add_argument("--repeats", type=int, default=1)
    args = p.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import fc_inputs as fi
    from . import fc

    prob = fi.config1() if args.problem == "2d" else fi.config2(int(args.problem))
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, precision=args.precision)
    B = fc.CP.from_factors(*prob.rhs())
    U = fc.CP(prob.d, prob.n, prob.max_rank)
    stream = torch.cuda.current_stream()
    for r in range(max(1, args.repeats)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps)
        e1.record(stream)
        e1.synchronize()
        print(f"{prob.label} precision={args.precision} solve {r}: status {info.status} "
              f"iters {info.iters} relres {info.relres:.2e} rank {U.rank} "
              f"max rank {info.max_rank_seen} truncations {info.trunc_calls} "
              f"{e0.elapsed_time(e1):.2f} ms", flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
