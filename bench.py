"""Benchmark: prox-grad iterations/s and time-to-converge of the Cov solver at
p = 65536, n = 32768 (X stored BF16, S FP32, lambda = (0.15, 0.05)).

A step is one whole solve from X resident in HBM: the Gram S = X^T X / n
(hpc_load_x) plus prox-grad iterations until ||dOmega||_F/||Omega||_F < 1e-6
(hpc_solve).  value = iterations of all timed steps / device time of those
steps; ms_per_step is the time-to-converge.  Inputs (X 4.3 GB, S 17 GB) are
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica of the workload on its GPU
(the solver does not shard); value sums the ranks' iterations over the
slowest rank's time.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "prox-grad iters/s, Cov solve at p=65536 n=32768 (time-to-converge = ms_per_step)"
UNIT = "iters/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained"), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_ready(self, timeout=5.0):
        """Block until nvidia-smi has printed its first sample, so that a short timed
        region starts with the sampler running."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_over_ranks(ms, iters, pg, device):
    """Slowest rank's time and the summed iterations of all ranks (replicas)."""
    if pg is None:
        return float(ms), float(iters)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.all_reduce(u, op=pg.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def measured_traffic(kernel, p, n, tag=""):
    """DRAM bytes per launch of `kernel` ("screen_pass", "gram" or "dense_grad") from the committed
    ncu summary (profiles/roofline_traffic.txt, 1-pass captures at the full
    workload); None when it was taken on other sizes, another version of the
    kernel's source, or (tag) another launch configuration of the kernel."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    srcs = {"screen_pass": "iterate.cu", "gram": "gram_tc.cu", "dense_grad": "adjoint.cu"}
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
        with open(os.path.join(ROOT, "paper_1710_10769_gb300", "csrc", srcs[kernel]), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != kv[f"{kernel}.src_sha256"]:
                return None
        if int(kv[f"{kernel}.p"]) != p or int(kv[f"{kernel}.n"]) != n:
            return None
        return float(kv[f"{kernel}.{tag}dram_bytes" if tag else f"{kernel}.dram_bytes"])
    except Exception:
        return None


def lemma31_flops(n, p, s, t, d):
    """Lemma 3.1's dominant flop counts of the paper's formulation (Sec. 3), with s
    prox-gradient iterations, t line-search trials per iteration and d nonzeros per row
    of the iterate:
      F_Cov = 2 n p^2 + 2 d p^2 (s t + 1)   (S once, then Omega S per trial),
      F_Obs = 2 n p^2 s + 2 d n p (s t + 1) (Z = Y X per iteration, Y = Omega X^T per trial),
    and the lemma's condition for Cov to be the cheaper, d/p < n / ((p - n) t) (its large-s
    limit; always true for p <= n)."""
    cov = 2.0 * n * p * p + 2.0 * d * p * p * (s * t + 1)
    obs = 2.0 * n * p * p * s + 2.0 * d * n * p * (s * t + 1)
    cheaper = True if p <= n else d / p < n / ((p - n) * t)
    return {"flops_cov": cov, "flops_obs": obs, "cov_cheaper": cheaper}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline_run(workload, X_host_cols, p_sample, max_seconds=25.0):
    """Time the FP64 oracle (as it stands: its CSR-iterate form of Alg. 2) on the leading
    p_sample x p_sample sub-problem of the workload: Gram, then the solve to the
    workload's stopping rule.

    Its Gram costs n p^2 and each of its iterations d p^2 (the candidate gradient over the
    whole matrix; d = nonzeros per row), so its rate at the full p is projected as
    rate(p_sample) * (p_sample / p)^2 -- a projection from a timed sample, labelled so.
    """
    import numpy as np

    import oracle

    t0 = time.perf_counter()
    S = oracle.gram_chunked(X_host_cols)
    threads = max(1, min(16, os.cpu_count() or 1))
    res = oracle.solve_sparse(S, workload.lambda1, workload.lambda2, eps=workload.eps, max_iter=100000,
                              block=512, threads=threads)
    dt = time.perf_counter() - t0
    rate_sample = res.iterations / dt
    scale = (p_sample / workload.p) ** 2
    try:
        from threadpoolctl import threadpool_info

        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [threads])
    except Exception:
        cores = os.cpu_count() or 1
    return {"value": rate_sample * scale, "unit": UNIT, "cores": int(cores), "kind": "oracle",
            "sample": (f"FP64 oracle (CSR form of Alg. 2) timed on the leading {p_sample}x{p_sample} sub-problem "
                       f"(same n={X_host_cols.shape[0]}, lambda, eps): Gram + {res.iterations} iterations in "
                       f"{dt:.1f} s = {rate_sample:.3f} iters/s; projected to p={workload.p} by "
                       f"({p_sample}/{workload.p})^2"),
            "seconds": dt, "iterations": res.iterations, "rate_sample": rate_sample}


def sample_subproblem(w, ps):
    """X (float64, the workload's storage values) of the leading ps x ps sub-problem of the
    workload's law: n samples of N(0, B^-1) with B = Omega0's leading ps x ps block (itself
    diagonally dominant), drawn on the CPU with the workload's seed."""
    import numpy as np

    from workloads import omega0_for, sample_x_cpu

    om = omega0_for(w)[:ps, :ps]
    workers = max(1, min(8, os.cpu_count() or 1))
    return sample_x_cpu(om, w.n, w.seed, workers=workers, chunk=256, x_dtype=w.x_dtype).astype(np.float64)


def _oracle_cores():
    try:
        from threadpoolctl import threadpool_info

        return int(max([d.get("num_threads", 1) for d in threadpool_info()] + [1]))
    except Exception:
        return os.cpu_count() or 1


def _line(metric, value, unit, ms, args, higher, dtype, config, roofline, clocks, launches, cpu, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": higher, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded generator)", "config": config, "roofline": roofline, "clocks": clocks,
            "e2e": None, "gpu_launches": launches, "cpu_baseline": cpu}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_row(args):
    """One line per further row of the hot path, on its own workload:
    path    -- the 32-point lambda1 path of path_p8192 (warm starts, one graph launch);
    batch   -- the 16 uneven problems p = 1024 k, solved as one graph launch;
    adjoint -- dL/dOmega, dL/dX and the hypergradient at p = 16384 after a solve;
    obs     -- the Obs variant (Z = Y^T X / n on tensor cores) on fp32_p16384.
    Each carries the FP64 oracle timed on a bounded sample of the same workload."""
    import numpy as np
    import torch

    import oracle
    import paper_1710_10769_gb300 as hpc
    from workloads import (BATCH_PROBLEMS, PATH_LAMBDA1, PATH_LAMBDA2, WORKLOADS, make_x, omega0_for,
                           sample_x_cpu, sample_x_cuda, cast_x, HELDOUT_STREAM)

    hbm, bf16, bf16_sus, peak_src = _peaks()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()

    if args.row == "path":
        w = WORKLOADS["path_p8192"]
        lam = sorted(PATH_LAMBDA1, reverse=True)
        X = make_x(w, device="cuda")
        s = hpc.Solver(X, lam[0], PATH_LAMBDA2, eps=w.eps, max_iter=100000, device_loop=args.device_loop)
        if args.fused_tail is not None:
            s.set_tuning(fused_tail=args.fused_tail)
        for _ in range(args.warmup):
            s.load_x(X)
            s.solve_path(lam, PATH_LAMBDA2, return_estimates=False)
        ms, its, it_ms = 0.0, 0, 0.0
        with ClockSampler(0) as clk:
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.load_x(X)
                pts, _ = s.solve_path(lam, PATH_LAMBDA2, return_estimates=False)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                its += sum(q["iterations"] for q in pts)
                it_ms += sum(q["ms"] for q in pts)
        p = w.p
        t_it = it_ms / its / 1000.0
        # An iteration is a chain of dependent, latency-bound steps (bound screening
        # reads a few MB of S; the candidate, line-search and accept steps touch the
        # candidate structure only): no bandwidth or tensor roofline bounds it.  For
        # scale, the time one full read of S would take at the copy figure.
        roof = {"kernel": "path iteration (screening, candidates, line search, accept)",
                "bound": "latency (dependent steps)", "iteration_us": t_it * 1e6,
                "full_S_read_us_at_peak": 4.0 * p * p / (hbm * 1e9) * 1e6, "peak_source": peak_src,
                "per_kernel": "profiles/path_p8192_launches.md"}
        cpu = None
        if not args.no_cpu:
            # the oracle: warm-started path on the leading 1024 x 1024 sub-problem, first points
            ps = min(1024, p)
            Xs = sample_x_cpu(omega0_for(w)[:ps, :ps], w.n, w.seed).astype(np.float32).astype(np.float64)
            t0 = time.perf_counter()
            S = oracle.gram(Xs)
            om, oits, npts = None, 0, 0
            for l1 in lam:
                r = oracle.solve(S, l1, PATH_LAMBDA2, eps=w.eps, max_iter=100000, omega0=om)
                om, oits, npts = r.omega, oits + r.iterations, npts + 1
                if time.perf_counter() - t0 > 20.0:
                    break
            dt = time.perf_counter() - t0
            cpu = {"value": oits / dt * (ps / p) ** 2, "unit": "iters/s", "cores": _oracle_cores(), "kind": "oracle",
                   "sample": f"FP64 oracle path over the first {npts} lambda1 points (warm starts, {oits} iterations, "
                             f"{dt:.1f} s) of the leading {ps}x{ps} sub-problem, rate scaled by ({ps}/{p})^2"}
        _line("lambda1 path iters/s, 32 points on p=8192 n=4096 (ms_per_step = load + whole path)", its / (ms / 1000),
              "iters/s", ms / args.steps, args, True, "f32",
              {"workload": "path_p8192", "p": p, "n": w.n, "points": len(lam), "lambda2": PATH_LAMBDA2,
               "gram_precision": s.precision_name(), "fused_tail": int(s.get_tuning()["fused_tail"]),
               "loop": "one graph launch per path" if args.device_loop else "host-driven"},
              roof, clk.summary(), None, cpu, iterations_per_step=its // args.steps,
              iteration_ms=t_it * 1000)
        s.close()
        return 0

    if args.row == "select":
        # model selection over the 32-point lambda1 grid of the path workload: the path, the
        # held-out loss of every point on the device, support recovery against Omega0
        from paper_1710_10769_gb300.selection import select_lambda1

        w = WORKLOADS["path_p8192"]
        lam = sorted(PATH_LAMBDA1, reverse=True)
        om0 = omega0_for(w)
        X = make_x(w, device="cuda")
        Xv = cast_x(sample_x_cuda(om0, w.n // 2, w.seed, stream=HELDOUT_STREAM), "f32")
        s = hpc.Solver(X, lam[0], PATH_LAMBDA2, eps=w.eps, max_iter=100000)
        for _ in range(args.warmup):
            s.load_x(X)
            select_lambda1(s, Xv, lam, PATH_LAMBDA2)
        ms = 0.0
        with ClockSampler(0) as clk:
            for _ in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.load_x(X)
                sel = select_lambda1(s, Xv, lam, PATH_LAMBDA2)
                torch.cuda.synchronize()
                ms += (time.perf_counter() - t0) * 1000.0
        from paper_1710_10769_gb300.selection import support_recovery

        s.load_x(X)
        sel = select_lambda1(s, Xv, lam, PATH_LAMBDA2, truth=om0)
        table = [{"lambda1": l1, "heldout": hl, "nnz": pt["nnz"], "iterations": pt["iterations"],
                  "ppv": rc["ppv"], "fdr": rc["fdr"], "tpr": rc["tpr"], "pairs": rc["pairs"]}
                 for l1, hl, pt, rc in zip(sel["lambda1"], sel["heldout"], sel["points"], sel["recovery"])]
        best_ppv = max(table, key=lambda r: (r["ppv"] if r["tpr"] > 0 else 0, r["tpr"]))
        _line("model selection over 32 lambda1 on p=8192 n=4096 (held-out n=2048): ms per selection", ms / args.steps,
              "ms", ms / args.steps, args, False, "f32",
              {"workload": "path_p8192", "p": w.p, "n": w.n, "n_val": w.n // 2, "points": len(lam),
               "lambda2": PATH_LAMBDA2, "timing": "host clock around load + path + held-out losses"},
              None, clk.summary(), None, None, selected={"lambda1": sel["lambda1"][sel["best"]], **table[sel["best"]]},
              best_ppv_point=best_ppv, table=table)
        s.close()
        return 0

    if args.row == "crossover":
        # One GPU's Fig. 2 (Section 4): p = 40000, n = 100 ... 12800, chain and random graphs,
        # time to converge of Cov (Gram + iterations) and Obs (Z every iteration), with
        # lambda1 = sqrt(2 log p / n) (the noise level of S's off-diagonal entries), lambda2 = 0.1.
        from workloads import omega0_banded, omega0_random

        p = 40000
        ns = [100, 200, 400, 800, 1600, 3200, 6400, 12800]
        rows = []
        with ClockSampler(0) as clk:
            for graph in ("chain", "random"):
                om0 = omega0_banded(p, 1, 5) if graph == "chain" else omega0_random(p, 8.0, 5)
                for n in ns:
                    X = cast_x(sample_x_cuda(om0, n, 5), "f32")
                    lam1 = math.sqrt(2.0 * math.log(p) / n)
                    rec = {"graph": graph, "n": n, "lambda1": lam1}
                    for vname, v in (("cov", hpc.COV), ("obs", hpc.OBS)):
                        s = hpc.Solver(None, lam1, 0.1, variant=v, n=n, p=p, xdtype=hpc.F32, eps=1e-6,
                                       max_iter=20000, precision=hpc.PREC_FP32 if v == hpc.OBS else hpc.PREC_BF16X3)
                        for rep in range(2):            # the first is a warm-up (graph capture, first-use costs)
                            torch.cuda.synchronize()
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            e0.record(stream)
                            s.load_x(X)
                            st = s.solve().as_dict()
                            e1.record(stream)
                            torch.cuda.synchronize()
                        rec[vname] = {"ms": e0.elapsed_time(e1), "iterations": st["iterations"],
                                      "trials": st["ls_trials"], "nnz": st["nnz"], "status": st["status"]}
                        s.close()
                    sc = rec["cov"]["iterations"]
                    tc = rec["cov"]["trials"] / max(sc, 1)
                    dc = rec["cov"]["nnz"] / p
                    auto, _, _ = hpc.choose_variant(n, p)
                    meas, cc, co = hpc.choose_variant(n, p, sc, tc, dc, 0.0)
                    rec["faster"] = "cov" if rec["cov"]["ms"] < rec["obs"]["ms"] else "obs"
                    rec["auto"] = "cov" if auto == hpc.COV else "obs"
                    rec["lemma_with_measured_s_t_d"] = "cov" if meas == hpc.COV else "obs"
                    rec["lemma_flops"] = lemma31_flops(n, p, sc, tc, dc)
                    rows.append(rec)
                    print(json.dumps(rec), file=sys.stderr, flush=True)
                    del X
                    torch.cuda.empty_cache()
        agree = sum(r["auto"] == r["faster"] for r in rows)
        total_ms = sum(min(r["cov"]["ms"], r["obs"]["ms"]) for r in rows)
        _line("Cov vs Obs crossover at p=40000, n=100..12800 (ms of the AUTO choice summed over the sweep)",
              sum(r[r["auto"]]["ms"] for r in rows), "ms", total_ms, args, False, "f32",
              {"workload": "crossover_p40000", "p": p, "n": ns, "graphs": ["chain (bandwidth 1)", "random (d = 8)"],
               "lambda1": "sqrt(2 log p / n)", "lambda2": 0.1, "timing": "CUDA events around load + solve"},
              None, clk.summary(), None, None, auto_picks_faster=f"{agree}/{len(rows)}", sweep=rows)
        return 0

    if args.row == "chain":
        # The paper's headline shape on one GPU (Abstract; Section 4, Fig. 4a; Table 1): chain
        # graph (bandwidth 1), n = 100, p up to 1.28 million, Obs variant (Z = Y X / n on the
        # tensor cores every iteration, no p x p array anywhere).  lambda1 = sqrt(2 log p / n),
        # the noise level of S's off-diagonal entries (the crossover row's rule), which puts
        # the estimate's average degree near the chain's 2 -- the paper compares equally
        # sparse estimates; the degree reached is reported.
        from paper_1710_10769_gb300.selection import support_recovery
        from workloads import omega0_banded

        n, lam2, seed = 100, 0.1, 5
        ps = [int(v) for v in args.chain_p.split(",")]
        rows = []
        with ClockSampler(0) as clk:
            for i, p in enumerate(ps):
                om0 = omega0_banded(p, 1, seed)
                X = cast_x(sample_x_cuda(om0, n, seed), "f32")
                lam1 = math.sqrt(2.0 * math.log(p) / n)
                s = hpc.Solver(None, lam1, lam2, variant=hpc.OBS, n=n, p=p, xdtype=hpc.F32,
                               precision=hpc.PREC_FP32, eps=1e-6, max_iter=5000, timing=1,
                               device_loop=args.device_loop)
                if i == 0:                      # first use of the kernels and the graph capture
                    s.load_x(X)
                    s.solve()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.load_x(X)
                st = s.solve().as_dict()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                est = s.get_omega().to_scipy(p)
                rec = support_recovery(est, om0)
                info = s.info()
                npairs = ((p + 127) // 128) * ((p + 127) // 128 + 1) // 2
                per = st["ms_grad_pass"] / max(st["grad_pass_launches"], 1)
                kdim = (n + 63) // 64 * 64
                # tensor work of one Z pass: both tiles of every block pair at the padded K, three
                # BF16 products each (BF16X3)
                tf = 2.0 * 2 * npairs * 128 * 128 * kdim * 3 / (per / 1000.0) / 1e12
                r = {"p": p, "n": n, "lambda1": lam1, "lambda2": lam2, "ms_to_converge": ms,
                     "iterations": st["iterations"], "ls_trials": st["ls_trials"], "status": st["status"],
                     "nnz": st["nnz"], "avg_degree": (st["nnz"] - p) / p, "ppv": rec["ppv"], "tpr": rec["tpr"],
                     "ms_z_pass": per, "z_pass_share": st["ms_grad_pass"] / ms,
                     "z_pass_tflops_bf16_equiv": tf, "z_pass_frac_of_bf16": tf / (bf16_sus if bf16_sus else bf16),
                     "device_bytes": info.device_bytes, "p_squared_fp32_bytes": 4 * p * p,
                     "parameters": p * (p + 1) // 2, "z_precision": s.precision_name()}
                rows.append(r)
                print(json.dumps(r), file=sys.stderr, flush=True)
                s.close()
                del X
                torch.cuda.empty_cache()
        big = rows[-1]
        roof = {"kernel": "k_obs_pair (Z pass)", "bound": "tensor", "achieved": big["z_pass_tflops_bf16_equiv"],
                "peak": bf16_sus if bf16_sus else bf16, "unit": "TFLOP/s", "frac": big["z_pass_frac_of_bf16"],
                "traffic": None, "peak_source": f"{peak_src} (bf16 sustained; 3 BF16 products per element counted)"}
        _line(f"Obs time to converge, chain graph, n=100, p={big['p']}", big["ms_to_converge"] / 1000.0, "s",
              big["ms_to_converge"], args, False, "f32",
              {"workload": f"chain_n100_p{big['p']}", "variant": "obs", "graph": "chain (bandwidth 1)", "n": n,
               "p": ps, "lambda1": "sqrt(2 log p / n)", "lambda2": lam2, "eps": 1e-6,
               "timing": "CUDA events around load_x + solve, one cold solve per p"},
              roof, clk.summary(), None, None, sweep=rows)
        return 0

    if args.row == "gram":
        # The tensor-core Gram of the headline workload under every tile order the autotuner
        # chooses from (band of row blocks x tile schedule), block maxima on: one load per
        # setting, in a fixed order, after one warm-up load.  Timed with the library's CUDA
        # events around the Gram kernel; launch k of k_gram_tc_persist (after the warm-up)
        # is setting k of the list.
        w = WORKLOADS[args.workload]
        X = make_x(w, device="cuda")
        s = hpc.Solver(None, w.lambda1, w.lambda2, n=w.n, p=w.p,
                       xdtype={"bf16": hpc.BF16, "f32": hpc.F32}[w.x_dtype], precision=hpc.PREC_AUTO,
                       eps=w.eps, max_iter=10, timing=1)
        s.load_x(X)
        flops = float(w.n) * w.p * (w.p + 1)
        peak = bf16_sus if bf16_sus else bf16
        sweep = []
        with ClockSampler(0) as clk:
            for band in (2, 4, 8, 16, 32, 64):
                for sched in (1, 0):
                    s.set_tuning(gram_band=band, gram_schedule=sched, gram_maxima=1)
                    s.load_x(X)
                    st = s.iterate(0).as_dict()
                    ms = st["ms_gram_kernel"]
                    sweep.append({"band": band, "schedule": sched, "ms": ms,
                                  "tflops": flops / (ms / 1000.0) / 1e12,
                                  "traffic": measured_traffic("gram", w.p, w.n, f"band{band}.maxima1.sched{sched}.")})
        best = min(sweep, key=lambda r: r["ms"])
        roof = {"kernel": "gram", "bound": "tensor", "achieved": best["tflops"], "peak": peak, "unit": "TFLOP/s",
                "frac": best["tflops"] / peak, "traffic": best["traffic"],
                "peak_source": f"{peak_src} (bf16 sustained)", "nominal_peak": 2250.0,
                "frac_of_nominal": best["tflops"] / 2250.0}
        _line(f"tensor-core Gram TFLOP/s at p={w.p} n={w.n}, best tile order", best["tflops"], "TFLOP/s",
              best["ms"], args, True, w.x_dtype,
              {"workload": w.name, "p": w.p, "n": w.n, "gram_precision": s.precision_name(),
               "best": {"band": best["band"], "schedule": best["schedule"]}},
              roof, clk.summary(), len(sweep), None, sweep=sweep)
        s.close()
        return 0

    if args.row == "batch":
        Xs = [make_x(wk, device="cuda") for wk in BATCH_PROBLEMS]
        streams = [torch.cuda.Stream() for _ in BATCH_PROBLEMS]
        sv = [hpc.Solver(X, wk.lambda1, wk.lambda2, stream=st, eps=wk.eps, max_iter=100000)
              for X, wk, st in zip(Xs, BATCH_PROBLEMS, streams)]
        torch.cuda.synchronize()
        ms, its, per = 0.0, 0, None
        with ClockSampler(0) as clk:
            for k in range(args.warmup + args.steps):
                for sk, X in zip(sv, Xs):
                    sk.load_x(X)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = hpc.solve_batch(sv)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                if k >= args.warmup:
                    ms += 1000 * (t1 - t0)
                    its += sum(q["iterations"] for q in st)
                    per = [q["iterations"] for q in st]
        byt = sum(4.0 * wk.p * wk.p * it for wk, it in zip(BATCH_PROBLEMS, per)) * args.steps
        alg = byt / (ms / 1000) / 1e9
        # the problems' iterations run concurrently and are latency-bound (as in the
        # path); the rate at which one full read of S per iteration of every problem
        # would have to stream is given for scale only
        roof = {"kernel": "batched solves (concurrent iteration loops)", "bound": "latency (dependent steps)",
                "full_S_reads_equivalent_gbs": alg, "peak": hbm, "peak_source": peak_src,
                "note": "bound screening reads about 1% of each S per iteration, so this equivalent can exceed "
                        "the copy figure"}
        cpu = None
        if not args.no_cpu:
            # the oracle: full solves of the two smallest problems; seconds per iteration
            # scale as p^2 (Gram included), applied to every problem's iteration count
            t_it = []
            for wk in BATCH_PROBLEMS[:2]:
                Xc = make_x(wk, device="cpu").astype(np.float64)
                t0 = time.perf_counter()
                r = oracle.solve(oracle.gram(Xc), wk.lambda1, wk.lambda2, eps=wk.eps, max_iter=100000)
                t_it.append((time.perf_counter() - t0) / r.iterations / (wk.p / BATCH_PROBLEMS[0].p) ** 2)
            unit_t = sum(t_it) / len(t_it)
            t_all = sum(unit_t * (wk.p / BATCH_PROBLEMS[0].p) ** 2 * it for wk, it in zip(BATCH_PROBLEMS, per))
            cpu = {"value": sum(per) / t_all, "unit": "iters/s", "cores": _oracle_cores(), "kind": "oracle",
                   "sample": "FP64 oracle full solves of the p = 1024 and 2048 problems; seconds per iteration scaled "
                             "by (p/1024)^2 over the 16 problems' iteration counts"}
        _line("batched solve iters/s, 16 problems p=1024..16384 (ms_per_step = the batch, Gram excluded)",
              its / (ms / 1000), "iters/s", ms / args.steps, args, True, "f32",
              {"workload": "batch16", "p": [wk.p for wk in BATCH_PROBLEMS], "n": "p/2",
               "loop": "one graph, a branch per problem", "timing": "host clock, device synchronised"},
              roof, clk.summary(), None, cpu, iterations_per_problem=per)
        for sk in sv:
            sk.close()
        return 0

    if args.row == "adjoint":
        w = WORKLOADS["adjoint_p16384"]
        om0 = omega0_for(w)
        Xtr = cast_x(sample_x_cuda(om0, w.n, w.seed), "f32")
        Xva = cast_x(sample_x_cuda(om0, 2048, w.seed, stream=HELDOUT_STREAM), "f32")
        s = hpc.Solver(Xtr, w.lambda1, w.lambda2, precision=hpc.PREC_FP32, eps=w.eps, max_iter=100000)
        s.solve()
        for _ in range(args.warmup):
            s.backward(Xtr)
            s.hypergrad(Xva, tol=1e-10)
        # A step is ~2-3 ms: time at least args.steps of them and at least 0.4 s, so that
        # the clock sampler (200 ms period) sees the timed region.
        mb, mh, steps = 0.0, 0.0, 0
        with ClockSampler(0) as clk:
            clk.wait_ready()
            t_start = time.perf_counter()
            while steps < args.steps or time.perf_counter() - t_start < 0.4:
                steps += 1
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                s.backward(Xtr)
                e1.record(stream)
                d1, d2, info = s.hypergrad(Xva, tol=1e-10)
                e2.record(stream)
                torch.cuda.synchronize()
                mb += e0.elapsed_time(e1)
                mh += e1.elapsed_time(e2)
        args = argparse.Namespace(**{**vars(args), "steps": steps})
        p, n = w.p, w.n
        # The dominant kernel, k_dense_grad_pair (dL/dOmega), timed on its own: one
        # backward call with dL/dX off is the row-info kernel plus that kernel.  It must
        # read the p (p + 1) / 2 distinct FP32 elements of S once and write the p x p
        # FP32 G once: 4 p^2 + 2 p (p + 1) bytes.
        md = 0.0
        for _ in range(args.steps):
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record(stream)
            s.backward(Xtr, dx=False)
            e1.record(stream)
            torch.cuda.synchronize()
            md += e0.elapsed_time(e1)
        md /= args.steps
        byt = 4.0 * p * p + 2.0 * p * (p + 1)
        alg = byt / (md / 1000) / 1e9
        roof = {"kernel": "k_dense_grad_pair", "bound": "hbm", "achieved": alg, "peak": hbm, "unit": "GB/s",
                "frac": alg / hbm, "traffic": measured_traffic("dense_grad", p, n), "peak_source": peak_src,
                "ms": md, "algorithmic_bytes": byt,
                "note": "distinct S elements read once, G written once; the gathered S rows of the few "
                        "off-diagonal support entries are not counted"}
        cpu = None
        if not args.no_cpu:
            csr = s.get_omega().to_scipy(p)
            Xh, Xvh = Xtr.cpu().numpy(), Xva.cpu().numpy()
            t0 = time.perf_counter()
            oracle.hypergrad_sparse(Xh, Xvh, csr, w.lambda1, w.lambda2)
            dt = time.perf_counter() - t0
            cpu = {"value": dt * 1000, "unit": "ms", "cores": _oracle_cores(), "kind": "oracle",
                   "sample": f"FP64 sparse hypergradient at full size on the GPU's support ({csr.nnz} entries)"}
        _line("adjoint + hypergradient ms per step at p=16384 (n=4096 train, 2048 held out)",
              (mb + mh) / args.steps, "ms", (mb + mh) / args.steps, args, False, "f32",
              {"workload": "adjoint_p16384", "p": p, "n": n, "n_val": 2048, "lambda1": w.lambda1,
               "lambda2": w.lambda2},
              roof, clk.summary(), None, cpu, backward_ms=mb / args.steps, hypergrad_ms=mh / args.steps,
              cg_iterations=info["cg_iterations"])
        s.close()
        return 0

    if args.row == "obs":
        w = WORKLOADS["fp32_p16384"]
        X = make_x(w, device="cuda")
        s = hpc.Solver(X, w.lambda1, w.lambda2, variant=hpc.OBS, eps=w.eps, max_iter=100000,
                       device_loop=args.device_loop)
        for _ in range(args.warmup):
            s.load_x(X)
            s.solve()
        ms, its, gp, gpl, launches = 0.0, 0, 0.0, 0, 0
        with ClockSampler(0) as clk:
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.load_x(X)
                st = s.solve().as_dict()
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                its += st["iterations"]
                gp += st["ms_grad_pass"]
                gpl += st["grad_pass_launches"]
                launches += st["kernel_launches"]
        p, n = w.p, w.n
        # one gradient pass forms Z = Y^T X / n = Omega S, which is not symmetric: both
        # Z[I, J] and Z[J, I] of every block pair, 2 n p^2 flop; three BF16 products per
        # element (BF16X3): a third of the bf16 peak
        per = gp / max(gpl, 1) / 1000.0
        tf = 2.0 * n * p * p / per / 1e12
        pk = (bf16_sus if bf16_sus else bf16) / 3.0
        roof = {"kernel": "obs gradient pass (Z GEMM)", "bound": "tensor", "achieved": tf, "peak": pk,
                "unit": "TFLOP/s", "frac": tf / pk, "traffic": None,
                "peak_source": f"{peak_src} (bf16 sustained / 3, BF16X3)", "ms_per_launch": per * 1000}
        cpu = None
        if not args.no_cpu:
            ps = min(1024, p)
            Xs = sample_x_cpu(omega0_for(w)[:ps, :ps], n, w.seed).astype(np.float32).astype(np.float64)
            t0 = time.perf_counter()
            r = oracle.solve_obs(Xs, w.lambda1, w.lambda2, eps=w.eps, max_iter=100000)
            dt = time.perf_counter() - t0
            cpu = {"value": r.iterations / dt * (ps / p) ** 2, "unit": "iters/s", "cores": _oracle_cores(),
                   "kind": "oracle",
                   "sample": f"FP64 oracle Obs solve ({r.iterations} iterations, {dt:.1f} s) of the leading {ps}x{ps} "
                             f"sub-problem (same n), rate scaled by ({ps}/{p})^2"}
        _line("Obs prox-grad iters/s at p=16384 n=8192 (ms_per_step = load + solve)", its / (ms / 1000), "iters/s",
              ms / args.steps, args, True, "f32",
              {"workload": "fp32_p16384", "variant": "obs", "p": p, "n": n, "lambda1": w.lambda1,
               "lambda2": w.lambda2, "z_precision": s.precision_name()},
              roof, clk.summary(), launches, cpu, iterations_per_step=its // args.steps)
        s.close()
        return 0
    raise SystemExit(f"unknown row {args.row}")


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.  Each step is a
    bounded sample of the workload (its leading cpu_sample_p x cpu_sample_p sub-problem,
    Gram + solve); ms_per_step is that step's measured wall time, and value the rate
    projected to the full workload (cpu_baseline_run), on this arm's metric and unit."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from workloads import WORKLOADS

    w = WORKLOADS[args.workload]
    ps = min(args.cpu_sample_p, w.p)
    X = sample_subproblem(w, ps)
    recs = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline_run(w, X, ps)
        if k >= args.warmup:
            recs.append(r)
    secs = sum(r["seconds"] for r in recs)
    its = sum(r["iterations"] for r in recs)
    value = its / secs * (ps / w.p) ** 2
    line = {"impl": "reference", "metric": METRIC.replace("p=65536 n=32768", f"p={w.p} n={w.n}"), "value": value,
            "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / len(recs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "data": f"synthetic (seeded: {w.graph} SDD Omega0, rows of X ~ N(0, Omega0^-1))",
            "config": {"workload": w.name, "p": w.p, "n": w.n, "lambda1": w.lambda1, "lambda2": w.lambda2,
                       "eps": w.eps, "x_dtype": w.x_dtype},
            "projection": {"measured_on_p": ps, "measured_iters_per_s": its / secs,
                           "scale": (ps / w.p) ** 2,
                           "rule": "Gram n p^2 and iterations d p^2: rate(p) = rate(sample) (sample / p)^2",
                           "ms_per_step": "measured wall time of one sample step (Gram + solve)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": recs[-1]["cores"], "kind": "oracle",
                             "sample": recs[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bf16_p65536")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16x3", "tf32"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-FP32 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-sample-p", type=int, default=2048)
    ap.add_argument("--device-loop", type=int, default=1, choices=[0, 1],
                    help="1 (default): iterations run as one CUDA-graph launch per solve, the library's "
                         "default; the Gram is timed with CUDA events either way, the screening pass with "
                         "device timestamps in this mode (CUDA events with 0)")
    ap.add_argument("--compare-loops", type=int, default=1, choices=[0, 1],
                    help="also time one solve with the other loop driver")
    ap.add_argument("--x-dtype", default="workload", choices=["workload", "f32", "bf16"],
                    help="store X in this dtype instead of the workload's (profiling the one-product BF16 Gram "
                         "at sizes a full ncu capture allows)")
    ap.add_argument("--row", default=None,
                    choices=["path", "batch", "adjoint", "obs", "select", "crossover", "chain", "gram"],
                    help="time a further row of the hot path instead of the headline solve")
    ap.add_argument("--chain-p", default="80000,160000,320000,640000,1280000",
                    help="dimensions of the chain row (comma separated)")
    ap.add_argument("--screen-bounds", type=int, default=1, choices=[0, 1],
                    help="0: screen without the block-maxima bounds (same result; for comparison)")
    ap.add_argument("--fused-tail", type=int, default=None, choices=[0, 1],
                    help="form of each iteration's steps after the screening pass: 0, the chain of kernels; "
                         "1, one cooperative kernel (default: the library's)")
    ap.add_argument("--compare-tail", type=int, default=1, choices=[0, 1],
                    help="also time the iteration loop with the other form of the tail")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="pick the launch shapes with the library's autotuner before the warm-up")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.row:
        return run_row(args)

    import numpy as np
    import torch

    import paper_1710_10769_gb300 as hpc
    from workloads import WORKLOADS, make_x

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    w = WORKLOADS[args.workload]
    prec = {"auto": hpc.PREC_AUTO, "fp32": hpc.PREC_FP32, "bf16x3": hpc.PREC_BF16X3, "tf32": hpc.PREC_TF32}[
        args.precision]
    X = make_x(w, device="cuda")
    if args.x_dtype != "workload":
        import dataclasses

        w = dataclasses.replace(w, x_dtype=args.x_dtype)
        X = X.to(torch.bfloat16 if args.x_dtype == "bf16" else torch.float32)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    xdt = {"bf16": hpc.BF16, "f32": hpc.F32, "f64": hpc.F64}[w.x_dtype]
    f64 = w.x_dtype == "f64"
    # FP64 workloads solve in FP64 values with the FP64 Gram
    vopt = dict(value_dtype=hpc.F64) if f64 else {}
    if f64 and args.precision == "auto":
        prec = hpc.PREC_FP64
    solver = hpc.Solver(None, w.lambda1, w.lambda2, n=w.n, p=w.p, xdtype=xdt, precision=prec, eps=w.eps,
                        max_iter=100000, device_loop=args.device_loop, **vopt)

    tuning, tune_trials = solver.get_tuning(), []
    if args.autotune:
        # the Gram's band (reloads X), then the iteration knobs from a mid-solve iterate
        _, tr0 = solver.autotune(X, iters=0)
        solver.iterate(8)
        tuning, tr1 = solver.autotune(None, iters=3)
        tune_trials = tr0 + tr1
    if not args.screen_bounds:
        solver.set_tuning(screen_bounds=0)
        tuning = solver.get_tuning()
    if args.fused_tail is not None:
        solver.set_tuning(fused_tail=args.fused_tail)
        tuning = solver.get_tuning()

    def step(Xsrc):
        solver.load_x(Xsrc)
        st = solver.solve().as_dict()
        st["ms_gram_step"] = st["ms_gram_kernel"]
        st["ms_load_step"] = st["ms_gram"]
        return st

    for _ in range(args.warmup):
        step(X)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    recs = []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            recs.append(step(X))
        ev1.record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    iters = sum(r["iterations"] for r in recs)
    ms_all, iters_all = reduce_over_ranks(ms, iters, pg, "cuda")
    value = iters_all / (ms_all / 1000.0)

    # rooflines of the two kernels that take the step's time: the Gram (one launch per
    # step) and the screening pass (one per iteration); the line's "roofline" is the
    # one with more device time per step
    hbm, bf16, bf16_sus, peak_src = _peaks()
    gram_ms = sum(r["ms_gram_step"] for r in recs)
    scr_ms = sum(r["ms_grad_pass"] for r in recs)
    scr_launches = sum(r["grad_pass_launches"] for r in recs)
    p, n = w.p, w.n
    tensor_gram = solver.precision_used() in (hpc.PREC_BF16X3, hpc.PREC_TF32)
    flops = float(n) * p * (p + 1)                   # symmetric half of X^T X: n p (p+1) FMA-flops
    g_achieved = flops / (gram_ms / len(recs) / 1000.0) / 1e12
    if tensor_gram:
        # a long kernel inside a long step: the sustained bf16 peak; TF32 at half the bf16 rate
        g_peak = bf16_sus if bf16_sus else bf16
        if solver.precision_used() == hpc.PREC_TF32:
            g_peak = g_peak / 2.0
        g_bound, g_src = "tensor", f"{peak_src} (bf16 sustained)"
    else:
        g_peak = 152 * 128 * 2 * 2.07e9 / 1e12       # SIMT FP32 FMA peak at the max SM clock
        g_bound, g_src = "alu", "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    # the nominal dense bf16 rate of the part (2.25 PFLOP/s; TF32 half of it), for the
    # fraction of the tensor pipe's own peak beside the fraction of the measured figure
    g_nominal = (2250.0 / (2.0 if solver.precision_used() == hpc.PREC_TF32 else 1.0)) if tensor_gram else g_peak
    roof_gram = {"kernel": "gram", "bound": g_bound, "achieved": g_achieved, "peak": g_peak, "unit": "TFLOP/s",
                 "frac": g_achieved / g_peak, "peak_source": g_src,
                 "nominal_peak": g_nominal, "frac_of_nominal": g_achieved / g_nominal,
                 # the Gram's traffic depends on its tile-order band and on whether it writes the block maxima
                 "traffic": measured_traffic("gram", p, n, f"band{tuning['gram_band']}.maxima{tuning['gram_maxima']}."
                                                           f"sched{tuning['gram_schedule']}."),
                 "ms_per_launch": gram_ms / len(recs),
                 "load_ms_per_step": sum(r["ms_load_step"] for r in recs) / len(recs)}
    per = scr_ms / max(scr_launches, 1) / 1000.0
    # The screening pass reads the (row, column block) maxima of |S| and only the
    # segments of S whose bound can emit, so it has no fixed byte count: it is
    # reported by time, against the time one full read of S's distinct elements
    # would take at the measured copy bandwidth.
    uniq = 4.0 * p * (p + 1) / 2.0
    roof_scr = {"kernel": "screen_pass", "bound": "hbm (bound-pruned reads)", "ms_per_launch": per * 1000.0,
                "full_triangle_read_ms_at_peak": uniq / (hbm * 1e9) * 1000.0,
                "speedup_vs_full_triangle_read_at_peak": (uniq / (hbm * 1e9)) / per,
                # captured with the bounds on
                "traffic": measured_traffic("screen_pass", p, n) if args.screen_bounds else None,
                "peak_source": peak_src}
    roof = roof_gram if gram_ms >= scr_ms else roof_scr

    # end to end through the C ABI with host buffers: each step reads its X from pinned
    # host memory and copies the CSR result back.  Steps alternate between two pinned
    # buffers (same contents), as a pipeline over successive data sets would: the next
    # step's X is staged (hpc_prefetch_x: a copy-engine transfer during this step's
    # Gram, its panel transpose during this step's solve).  Step 0 reads its own X and
    # the last step stages nothing, so the region holds one transfer per step.  One
    # timed region over all steps, after an untimed step that sizes the buffers.
    e2e = None
    if args.e2e_steps > 0:
        bufs = [X.cpu().pin_memory(), X.cpu().pin_memory()]
        solver.load_x(bufs[0])
        solver.solve()
        solver.get_omega(np.float32)
        torch.cuda.synchronize()
        e2e_its, d2h, marks = 0, 0, []
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            if k + 1 < args.e2e_steps:
                solver.prefetch_x(bufs[(k + 1) % 2])
            solver.load_x(bufs[k % 2])
            st = solver.solve().as_dict()
            csr = solver.get_omega(np.float32)
            e2e_its += st["iterations"]
            d2h += csr.row_ptr.nbytes + csr.col.nbytes + csr.val.nbytes
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1000
        e2e = {"value": e2e_its / (e2e_ms / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(bufs[0].numel() * bufs[0].element_size()),
               "d2h_bytes_per_step": int(d2h // args.e2e_steps), "steps": args.e2e_steps,
               "overlap": "next step's X staged during this step (hpc_prefetch_x), two pinned buffers",
               "step_ms": [round(1000 * (b - a), 1) for a, b in zip([t0] + marks[:-1], marks)]}
        del bufs

    # the same step with the other loop driver (host-driven iterations vs one CUDA-graph
    # launch per solve), for comparison
    other = None
    if args.compare_loops and rank == 0:
        alt = hpc.Solver(None, w.lambda1, w.lambda2, n=w.n, p=w.p, xdtype=xdt, precision=prec, eps=w.eps,
                         max_iter=100000, device_loop=1 - args.device_loop, **vopt)
        alt.set_tuning(**tuning)
        alt.load_x(X)
        alt.solve()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        alt.load_x(X)
        ast = alt.solve().as_dict()
        e1.record(stream)
        torch.cuda.synchronize()
        other = {"device_loop": 1 - args.device_loop, "ms_per_step": e0.elapsed_time(e1),
                 "value": ast["iterations"] / (e0.elapsed_time(e1) / 1000.0), "iterations": ast["iterations"]}
        alt.close()

    # the iteration loop with the other form of the tail (the chain of kernels or the
    # one cooperative kernel), same data, best of three solves
    other_tail = None
    if args.compare_tail and rank == 0:
        flip = 1 - int(tuning.get("fused_tail", 0))
        solver.set_tuning(fused_tail=flip)
        runs = []
        for _ in range(4):
            solver.load_x(X)
            runs.append(solver.solve().as_dict())
        solver.set_tuning(fused_tail=1 - flip)
        best = min(runs[1:], key=lambda r: r["ms_total"])
        mine = min(recs, key=lambda r: r["ms_total"])
        other_tail = {"fused_tail": flip, "iterations": best["iterations"],
                      "iteration_loop_its": best["iterations"] / (best["ms_total"] / 1000.0),
                      "kernel_launches_per_iteration": best["kernel_launches"] / max(best["iterations"], 1),
                      "this_line": {"fused_tail": int(tuning.get("fused_tail", 0)),
                                    "iteration_loop_its_best_step": mine["iterations"] / (mine["ms_total"] / 1000.0),
                                    "kernel_launches_per_iteration": mine["kernel_launches"] /
                                    max(mine["iterations"], 1)}}

    plain, plain_est = None, None
    if not args.no_plain and solver.precision_used() not in (hpc.PREC_FP32, hpc.PREC_FP64) and rank == 0:
        ps = hpc.Solver(None, w.lambda1, w.lambda2, n=w.n, p=w.p, xdtype=xdt, precision=hpc.PREC_FP32, eps=w.eps,
                        max_iter=100000, device_loop=args.device_loop)
        ps.set_tuning(**tuning)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ps.load_x(X)
        pst = ps.solve().as_dict()
        e1.record(stream)
        torch.cuda.synchronize()
        om_plain = ps.get_omega()
        om_mixed = solver.get_omega()
        A = om_plain.to_scipy(p)
        B = om_mixed.to_scipy(p)
        plain = {"time_to_converge_ms": e0.elapsed_time(e1), "iterations": pst["iterations"],
                 "gram_ms": pst["ms_gram"], "rel_diff_vs_mixed": float(
                     math.sqrt((A - B).multiply(A - B).sum()) / math.sqrt(A.multiply(A).sum()))}
        plain_est = om_plain
        ps.close()

    # error against the cached FP64 reference of this workload (written once by
    # tests/golden/make_fullsize_refs.py from the oracle), when the repository holds one
    accuracy = None
    ref_file = os.path.join(ROOT, "tests", "golden", f"ref_{w.name}.npz")
    if rank == 0 and os.path.exists(ref_file):
        import scipy.sparse as sp

        z = np.load(ref_file, allow_pickle=False)
        R = sp.csr_matrix((z["data"], z["indices"], z["indptr"]), shape=(p, p))
        rn = math.sqrt(R.multiply(R).sum())

        def err(est):
            E = est.to_scipy(p).astype(np.float64)
            D = E - R
            pe, pr = (E != 0), (R != 0)
            return {"rel_fro": math.sqrt(D.multiply(D).sum()) / rn,
                    "support_differences": int((pe != pr).nnz), "nnz": int(E.nnz)}

        accuracy = {"reference": f"FP64 oracle fixed point (eps {float(z['eps']):g}, {int(z['iterations'])} iterations, "
                                 f"certified within {float(z['distance_bound_rel']):.2e} relative of the minimiser)",
                    "nnz_ref": int(R.nnz), "mixed": err(solver.get_omega())}
        if plain is not None:
            accuracy["plain_fp32"] = err(plain_est)
    cpu = None
    if not args.no_cpu and rank == 0:
        ps = min(args.cpu_sample_p, w.p)
        c = cpu_baseline_run(w, sample_subproblem(w, ps), ps)
        cpu = {k: c[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        gpu_launches = sum(r["kernel_launches"] for r in recs) + sum(1 for _ in recs)
        line = {
            "metric": METRIC.replace("p=65536 n=32768", f"p={p} n={n}"), "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if f64 else ("bf16" if (w.x_dtype == "bf16" and tensor_gram) else "f32"),
            "data": f"synthetic (seeded: {w.graph} SDD Omega0, rows of X ~ N(0, Omega0^-1))",
            "config": {"workload": w.name, "p": p, "n": n, "lambda1": w.lambda1, "lambda2": w.lambda2,
                       "eps": w.eps, "x_dtype": w.x_dtype, "s_dtype": "f64" if f64 else "f32",
                       "gram_precision": solver.precision_name(), "parallelism": f"replicas x{ws}",
                       "loop": "device (one CUDA graph per solve)" if args.device_loop else "host-driven",
                       "tuning": tuning, "autotuned": bool(args.autotune),
                       "l2": (f"inputs > L2 (X {X.numel() * X.element_size() / 1e9:.2f} GB, S {4 * (1 + f64) * p * p / 1e9:.2f} GB); no flush"
                              if (1 + f64) * 4 * p * p > 129e6 else "S fits in L2 (small latency-bound case); no flush")},
            "iterations_per_step": [r["iterations"] for r in recs],
            "ls_trials_per_step": [r["ls_trials"] for r in recs],
            "time_to_converge_ms": ms_all / args.steps,
            "gram_ms_per_step": gram_ms / len(recs),
            "load_ms_per_step": sum(r["ms_load_step"] for r in recs) / len(recs),
            "iteration_loop_its": iters / (sum(r["ms_total"] for r in recs) / 1000.0),
            "grad_pass_ms": scr_ms / max(scr_launches, 1),
            "final_nnz": recs[-1]["nnz"], "final_F": recs[-1]["F"],
            # the paper's cost model (Lemma 3.1) for this solve, for context: s and t are the
            # solve's own counts, d the final estimate's nonzeros per row (the lemma averages
            # d over every trial's iterate)
            "paper_model": dict(lemma31_flops(n, p, recs[-1]["iterations"],
                                              recs[-1]["ls_trials"] / max(recs[-1]["iterations"], 1),
                                              recs[-1]["nnz"] / p),
                                s=recs[-1]["iterations"], d="final nnz / p"),
            "roofline": roof, "roofline_kernels": [roof_gram, roof_scr], "clocks": clk.summary(), "e2e": e2e, "gpu_launches": gpu_launches,
            "cpu_baseline": cpu, "plain_fp32": plain, "accuracy_vs_fp64_reference": accuracy, "other_loop": other,
            "other_tail": other_tail,
            "autotune_trials": [(t["knob"], t["value"], round(t["ms"], 4)) for t in tune_trials],
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
