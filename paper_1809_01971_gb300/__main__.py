"""Command-line solve of control problems (beta^2 A^-alpha + gamma A^alpha) u = beta y_Omega
with seeded synthetic right-hand sides:

    python -m paper_1809_01971_gb300 --problem 5 --precision 2 --repeats 3
    python -m paper_1809_01971_gb300 --batch 0:8 --precision 2 --spectral

--problem k selects the k-th 3D n = 255 problem (alpha in {0.25, 0.5, 0.75} x gamma in
{1e-1, 1e-3}: four separable Gaussians + one grid sine mode), --problem 2d the 2D n = 63 one;
--batch a:b solves problems a .. b-1 of the 512-problem mixed batch (n in {127 .. 2047}) one
after another on one stream, at their 1e-6 settings.  --precision picks the contraction form
(0 FP64, 1 double-float FP32, 2 tensor-core digit products).  Prints the PCG summary and the
device time of each solve (CUDA events).
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    p = argparse.ArgumentParser(prog="python -m paper_1809_01971_gb300")
    p.add_argument("--problem", default="5", help="0..5 (3D, n=255) or 2d (n=63)")
    p.add_argument("--batch", default=None, help="a:b, problems of the mixed batch")
    p.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    p.add_argument("--spectral", action="store_true")
    p.add_argument("--repeats", type=int, default=1)
    args = p.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import fc_inputs as fi
    from . import fc

    if args.batch:
        a, b = (int(x) for x in args.batch.split(":"))
        probs = [fi.config4(i) for i in range(a, b)]
    else:
        probs = [fi.config1() if args.problem == "2d" else fi.config2(int(args.problem))]
    stream = torch.cuda.current_stream()
    # set-up of every problem first; the solves run inside the NVTX range "fc_solve" (a
    # profiler can select them with it)
    work = []
    for prob in probs:
        h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                        max_rank=prob.max_rank, max_tucker=prob.max_tucker,
                        precision=args.precision)
        work.append((prob, h, fc.CP.from_factors(*prob.rhs()), fc.CP(prob.d, prob.n, prob.max_rank)))
    torch.cuda.synchronize()
    for prob, h, B, U in work:
        for r in range(max(1, args.repeats)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("fc_solve")
            e0.record(stream)
            info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, spectral=args.spectral,
                               stall=3 if args.batch else 0, raise_on_fail=False)
            e1.record(stream)
            e1.synchronize()
            torch.cuda.nvtx.range_pop()
            print(f"{prob.label} precision={args.precision} solve {r}: status {info.status} "
                  f"iters {info.iters} relres {info.relres:.2e} rank {U.rank} "
                  f"max rank {info.max_rank_seen} truncations {info.trunc_calls} "
                  f"{e0.elapsed_time(e1):.2f} ms", flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
