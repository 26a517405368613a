#!/usr/bin/env python
"""Throughput of the low-rank (CP) PCG control solve on one GB300, in 3D control solves/s.

Workload (one step): the six 3D problems d=3, n=255 (16.6M grid points each),
alpha in {0.25, 0.5, 0.75} x gamma in {1e-1, 1e-3}, beta = 1, right-hand side y_Omega =
4 seeded separable Gaussians + sin(pi x) sin(2 pi y) sin(3 pi z) (CP rank 5), truncation
eps = 1e-9, PCG tol = 1e-8, CP rank cap 192 (all six solutions within 1e-6 of the exact one).  Each problem's operator set-up (symbol and
preconditioner CP factors, workspace) is done once before timing, as a library user
would for repeated solves with one operator; the timed step is the full Algorithm 1
(PCG with RHOSVD truncation) for all six right-hand sides.

The step runs in each contraction form of the library (fc_setup precision 0: FP64; 1:
double-float FP32; 2: FP64-accurate digit products on the BF16 tensor cores), and form 2 also
with the spectral-resident iteration (fc_solve_opts.spectral); `forms` reports all of them,
and `value` is the fastest whose solutions are all within 1e-6 of the exact one
(`config.form`), `vs_plain_fp64` its ratio to the FP64 form.

`value`  : device-resident solves/s (CUDA events on the launching stream, L2 flushed
           between steps with a 512 MiB write, outside the events).
`e2e`    : the same through the public API with host buffers, in the reported form: every
           step copies the right-hand sides from pinned host memory and reads the
           solutions back.
Accuracy : after timing, every solution is compared with the library's full-format
           FP64 eigenbasis solve (16.6M points), and the largest relative L2 error is
           reported; a run where any form's error exceeds 1e-6 exits non-zero.
`--impl reference` times the CPU FP64 oracle on the same workload (one problem per
step, cycling) on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D control solves/s at rel-err<=1e-6 (CP-PCG, batched; fastest contraction form meeting the bound, vs plain FP64)"
UNIT = "solves/s"
WORKLOAD = "3d_n255_6problems_alpha{0.25,0.5,0.75}_gamma{1e-1,1e-3}_rank5rhs_tol1e-8_eps1e-9_cap192"
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--problems", type=int, default=6)
    p.add_argument("--max-err", type=float, default=1e-6,
                   help="exit status 3 when a solution's error vs the full solve exceeds this")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value over the ranks (the job's time is its slowest rank's)."""
    if world > 1:
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return float(x)


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time
    (weak scaling: each rank solves the full problem set)."""
    return units_per_rank * world / seconds


def problems(count):
    import fc_inputs as fi
    return [fi.config2(p % 6) for p in range(count)]


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_solve(prob):
    """One CP-PCG solve by the CPU FP64 oracle (symbols built as part of the solve)."""
    from oracle import pcg, quadrature as q
    fs = q.control_symbol(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, 1e-10)
    ps = q.precond_symbol(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, 24)
    return pcg.pcg(fs, ps, prob.rhs(), prob.eps, prob.tol, prob.max_rank)


def cpu_baseline(probs, budget_s=25.0):
    """Oracle solves/s on a bounded sample: whole solves of the workload's problems in order
    (alpha = 0.25 first, the quickest) until ~budget_s of CPU time has passed."""
    t0 = time.perf_counter()
    done = 0
    while done < len(probs):
        cpu_oracle_solve(probs[done])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of the {len(probs)} n=255 3D problems (in workload order, "
                      f"alpha=0.25 first: the quickest to converge), whole CP-PCG solves incl. "
                      f"symbol set-up, numpy/scipy FP64 with BLAS threads <= {cores}, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # one step = one oracle solve of the workload's first problem (alpha = 0.25, gamma = 0.1,
    # ~10 s on a few cores): a bounded sample, so that the whole run ends in minutes
    probs = problems(1)
    for i in range(args.warmup):
        cpu_oracle_solve(probs[0])
    t0 = time.perf_counter()
    for i in range(args.steps):
        cpu_oracle_solve(probs[0])
    dt = time.perf_counter() - t0
    v = args.steps / dt
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "step": "one oracle solve of problem 0 (alpha=0.25, gamma=0.1)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle solves of problem 0 of the workload "
                                       f"(the quickest of the six)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# FP64 peak of the chip from its unit counts and clock: 152 SMs x 2 FP64 FMA per clock per SM
# x 2 flop x 2.07 GHz (an FP64 probe on this part measured 1.19 TFLOP/s at 1.9-2.07 GHz).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# Dense BF16 tensor throughput of the GB300s, measured and sustained over seconds
# (cuBLAS 8192^3, MEASURED_PEAKS.json): the tensor-pipe peak of a kernel timed in a long step.
BF16_PEAK_SUSTAINED_TFLOPS = 1686.8
# Tensor-core contraction DRAM traffic per launch from one ncu capture; None when not captured
# for the current kernel.
TC_TRAFFIC_BYTES = None
# Eigen-solver DRAM traffic per launch (dram__bytes_read.sum + write) from one ncu capture of
# the current kernel (3-matrix launch of the n=255 solve); None when not captured for it.
EIG_TRAFFIC_BYTES = None


# (name, fc_setup precision, spectral-resident iteration, dtype, contractions)
FORMS = [("fp64", 0, False, "f64", "FP64 throughout"),
         ("df32", 1, False, "f32x2", "large contractions in double-float FP32 (hi+lo); rest FP64"),
         ("tc64", 2, False, "bf16-digits/f64",
          "large contractions as exact products of 8 fixed-point 7-bit digits on the BF16 "
          "tensor cores (tcgen05, FP32 TMEM accumulation, FP64-level error); rest FP64"),
         ("tc64_spectral", 2, True, "bf16-digits/f64",
          "as tc64, iterates kept in the DST-I eigenbasis (one transform at entry and exit)")]


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import paper_1809_01971_gb300 as fc

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    main_stream = torch.cuda.current_stream()
    probs = problems(args.problems)
    # independent problems: each rank solves the full six-problem set (weak scaling)
    Bs = [fc.CP.from_factors(*p.rhs(), device=dev) for p in probs]
    streams = [torch.cuda.Stream(device=dev) for _ in probs]
    tols = [p.tol for p in probs]
    epss = [p.eps for p in probs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        """Device time of fn() from CUDA events: start on the main stream, every problem
        stream waits on it, and the main stream waits for every problem stream at the end."""
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main_stream)
        for s_ in streams:
            s_.wait_event(e0)
        out = fn()
        for s_ in streams:
            main_stream.wait_stream(s_)
        e1.record(main_stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # accuracy reference: the library's full-format FP64 eigenbasis solve of every problem
    nn = probs[0].n ** 3
    full_b = torch.empty(nn, dtype=torch.float64, device=dev)
    tmp = torch.empty_like(full_b)
    full_u = []
    href = [fc.fc_setup(p.n, p.d, p.alpha, p.beta, p.gamma, p.eps, max_rank=p.max_rank)
            for p in probs]
    for p, h, B in zip(probs, href, Bs):
        fc.fc_to_full(h, B, out=full_b)          # column-major n^3
        u = torch.empty_like(full_b)
        fc.fc_full_solve(h, full_b, u, tmp)
        full_u.append(u)

    sampler = ClockSampler(local)
    sampler.start()
    results = {}
    handles = {0: href}
    for form, (fname, prec, spectral, _, _) in enumerate(FORMS):
        if prec not in handles:
            handles[prec] = [fc.fc_setup(p.n, p.d, p.alpha, p.beta, p.gamma, p.eps,
                                         max_rank=p.max_rank, precision=prec) for p in probs]
        hs = handles[prec]
        Us = [fc.CP(p.d, p.n, p.max_rank, device=dev) for p in probs]

        def step(hs=hs, Us=Us, spectral=spectral):
            # the step's problems run concurrently, one stream each (fc_solve_batched)
            return fc.fc_solve_batched(hs, Bs, Us, tol=tols, eps=epss, spectral=spectral,
                                       stream=main_stream)

        for _ in range(args.warmup):
            step()
        barrier()
        fc.fc_prof_enable(fc.fc.PROF_JACOBI)
        launches0 = fc.fc_launch_count()
        times, iters = [], []
        for _ in range(args.steps):
            ms, infos = timed(step)
            times.append(ms)
            iters.append([i.iters for i in infos])
        launches = fc.fc_launch_count() - launches0
        prof = fc.fc_prof_read()
        barrier()
        t_total = max_over_ranks(sum(times) / 1e3, world, dev)
        err = 0.0
        for h, U, u in zip(hs, Us, full_u):
            fc.fc_to_full(h, U, out=tmp)
            err = max(err, float(torch.linalg.norm(tmp - u) / torch.linalg.norm(u)))
        tc_prof = None
        if fname == "tc64":
            # the tensor-core contraction class, instrumented over extra (untimed) steps
            fc.fc_prof_enable(fc.fc.PROF_TC)
            tc_times = [timed(step)[0] for _ in range(args.steps)]
            tc_prof = fc.fc_prof_read() + (sum(tc_times),)
            barrier()
        results[form] = {"hs": hs, "Us": Us, "step": step, "t_total": t_total,
                         "value": job_rate(len(probs) * args.steps, world, t_total),
                         "launches": launches, "prof": prof, "iters": iters[-1], "err": err,
                         "tc_prof": tc_prof}
    clocks = sampler.stop()

    ok = [f for f in results if results[f]["err"] <= args.max_err]
    best = max(ok, key=lambda f: results[f]["value"]) if ok else 0
    R = results[best]
    value, t_total = R["value"], R["t_total"]
    solves = len(probs) * args.steps * world

    # the FP64 problems one after another on one stream (context for the batched number)
    hs0, Us0 = results[0]["hs"], results[0]["Us"]

    def step_sequential():
        return [fc.fc_solve(h, B, U, tol=p.tol, eps=p.eps, stream=main_stream)
                for p, h, B, U in zip(probs, hs0, Bs, Us0)]

    seq_steps = max(1, args.steps // 2)
    seq_ms = sum(timed(step_sequential)[0] for _ in range(seq_steps))
    seq_value = len(probs) * seq_steps / (seq_ms / 1e3)

    # end to end through the public API with host buffers, in the reported form
    hsb, Usb = R["hs"], R["Us"]
    host_in = []
    for p in probs:
        xi, U = p.rhs()
        host_in.append((torch.tensor(xi).pin_memory(),
                        torch.tensor(np.stack([u.T for u in U])).pin_memory()))
    host_out = [(torch.empty(p.max_rank, dtype=torch.float64).pin_memory(),
                 torch.empty(p.d, p.max_rank, p.n, dtype=torch.float64).pin_memory()) for p in probs]
    h2d = sum(a.numel() * 8 + b.numel() * 8 for a, b in host_in)
    d2h = sum(a.numel() * 8 + b.numel() * 8 for a, b in host_out)

    def e2e_step():
        for (xi_h, U_h), p, B, s_ in zip(host_in, probs, Bs, streams):
            R_ = xi_h.numel()
            with torch.cuda.stream(s_):
                B.xi[:R_].copy_(xi_h, non_blocking=True)
                B.U[:, :R_, :p.n].copy_(U_h, non_blocking=True)
            B.rank = R_
        fc.fc_solve_batched(hsb, Bs, Usb, tol=tols, eps=epss, spectral=FORMS[best][2],
                            stream=main_stream)
        for (xo, Uo), p, U, s_ in zip(host_out, probs, Usb, streams):
            with torch.cuda.stream(s_):
                xo.copy_(U.xi[:p.max_rank], non_blocking=True)
                Uo.copy_(U.U[:, :p.max_rank, :p.n], non_blocking=True)

    timed(e2e_step)
    e2e_times = []
    barrier()
    for _ in range(args.steps):
        e2e_times.append(timed(e2e_step)[0])
    barrier()
    e2e_value = job_rate(len(probs) * args.steps, world, max_over_ranks(sum(e2e_times) / 1e3, world, dev))

    roofline = None
    jac_n, jac_ms, jac_work = R["prof"]
    if jac_n > 0 and jac_ms > 0:
        achieved = jac_work / jac_n / (jac_ms / jac_n * 1e-3) / 1e12     # TFLOP/s
        peak = FP64_PEAK_GFLOPS / 1e3
        roofline = {"kernel": "gjacobi_kernel (graded eigen-solves of the RHOSVD: FP32 Jacobi "
                              "sweeps, FP64 orthonormalisation)",
                    "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": EIG_TRAFFIC_BYTES,
                    "peak_kind": "FP64, derived: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
                    "work": "9 c^3 flop per c x c matrix (textbook dense eigen-solve count)",
                    "launches": jac_n, "avg_launch_us": 1e3 * jac_ms / jac_n,
                    "event_ms_over_step_ms": jac_ms / (t_total * 1e3),
                    "note": "launches overlap across the problem streams, so summed event time can exceed step time"}
    roofline_tc = None
    if results[2]["tc_prof"] and results[2]["tc_prof"][0] > 0:    # FORMS[2] = tc64
        tn, tms, twork, tstep_ms = results[2]["tc_prof"]
        achieved = twork / tn / (tms / tn * 1e-3) / 1e12
        peak = BF16_PEAK_SUSTAINED_TFLOPS
        roofline_tc = {"kernel": "gemm_tc_kernel (FP64 contractions of the tc64 form as BF16 "
                                 "digit-pair MMAs on tcgen05, TMEM accumulators)",
                       "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak, "traffic": TC_TRAFFIC_BYTES,
                       "peak_kind": "measured BF16 dense, sustained (MEASURED_PEAKS.json)",
                       "work": "BF16 MMA flops issued: 36 digit pairs x 2 x 128 x N_tile per K",
                       "launches": tn, "avg_launch_us": 1e3 * tms / tn,
                       "event_ms_over_step_ms": tms / tstep_ms}
    if rank == 0:
        name, _, _, dtype, what = FORMS[best]
        forms = {FORMS[f][0]: {"value": results[f]["value"], "unit": UNIT,
                               "ms_per_step": 1e3 * results[f]["t_total"] / args.steps,
                               "max_rel_err_vs_full": results[f]["err"],
                               "pcg_iters": results[f]["iters"],
                               "gpu_launches": int(results[f]["launches"]),
                               "contractions": FORMS[f][4]} for f in results}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": WORKLOAD, "problems_per_step": len(probs),
                           "form": name,
                           "l2": "flushed between steps (512 MiB write, untimed)",
                           "setup": "per operator, before timing",
                           "concurrency": "fc_solve_batched: one stream per problem, up to 16 host threads",
                           "work_queues": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"),
                           "pcg_iters": R["iters"]},
                "forms": forms,
                "vs_plain_fp64": value / results[0]["value"],
                "sequential_fp64_value": seq_value,
                "max_rel_err_vs_full": R["err"],
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(R["launches"]),
                "clocks": clocks,
                "roofline": roofline,
                "roofline_tc": roofline_tc,
                "cpu_baseline": None}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(probs)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0 if all(results[f]["err"] <= args.max_err for f in results) else 3


if __name__ == "__main__":
    sys.exit(main())
