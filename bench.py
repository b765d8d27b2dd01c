"""Benchmark: time-to-solution of the Helmholtz DD solve at k=200, ~20 ppwl (N=640, 8x8
subdomains, overlap 2, centre point source + seeded Gaussian bump), outer FGMRES to relative
residual 1e-6, inner deflated GMRES to 1e-2 in complex64 (FP32 accumulation), coarse E and
outer Arnoldi in FP64.

One step = one full solve (every step of the path) on inputs already resident in HBM.  Prints one
JSON line.  `--impl reference` times the CPU oracle instead (bounded sample per step).

Besides the default form (the line's value) the line carries, under "forms", the plain FP64 GPU
method (complex128 inner, all-FP64 outer) and the learned-warm-start form, each timed with fewer
steps, and for every form its error against the oracle's stored solve of the same workload
(tests/golden/<workload>_oracle_x.npy, written by an oracle-only script).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "time-to-solution at rel-res 1e-6 (k=200, 20 ppwl); subdomain-solve GB/s vs peak"
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12     # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TINSTR = 152 * 128 * 2.070e9 / 1e12    # 152 SMs x 128 FP32 lanes x 2.07 GHz (instructions)
# the library's default outer Arnoldi: delayed CGS2 with double-FP32 dots and updates
OUTER_DF = "dcgs2-df32"
L2_FLUSH_BYTES = 512 << 20                      # > 129 MB L2
# DRAM bytes (read + written) per algorithmic byte of a kernel family, from one ncu capture of its
# kernels at outer iteration 200 of the k=200 solve (profiles/); their traffic grows with the
# basis vectors read, so the ratio scales that capture to the average launch of a k=200 run.
# Keyed by (family, double-FP32 dots on); a family whose kernels changed since their capture has
# no entry, and the roofline's traffic field is then null.
TRAFFIC_PER_ALG = {
    # k_odots + k_oupdate (FP64 dots): 1.9827 + 4.0434 GB against 1.9763 + 3.9525 GB
    ("outer_cgs2_fp64", False): (1.982693 + 4.043380) / (1.976274 + 3.952547),
    # k_oupdate without dots (double-FP32 dots on): 2.0608 + 0.0061 GB against 1.9828 GB
    ("outer_cgs2_fp64", True): (2.060811 + 0.006137) / ((201 * 24 + 32) * 408321 / 1e9),
    # k_odots2_df<1> (delayed CGS2 with biased first-pass dots, step 199): 1.3200 + 0.0052 GB
    # against 1.3197 GB
    ("outer_dots_df32", True): (1.320033 + 0.005162) / ((200 * 16 + 32) * 408321 / 1e9),
    # k_oupdate_dcgs (step 199): 1.3134 + 0.0189 GB against 1.3360 GB
    ("outer_update_df32", True): (1.313391 + 0.018886) / ((199 * 16 + 88) * 408321 / 1e9),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank, int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value: float, device: str) -> float:
    """The largest value over the ranks of the process group (the slowest replica sets the step
    time); the value itself without a group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def oracle_sample(w, outer_its: int, threads: int = 0):
    """Time the CPU oracle on the first `outer_its` outer iterations of workload w."""
    import oracle
    if threads:
        oracle.set_threads(threads)
    p = oracle.from_workload(w)
    f = p.rhs(w.rhs[0])
    t0 = time.perf_counter()
    _, st = p.solve(f, outer_tol=w.outer_tol, inner_tol=w.inner_tol, outer_maxit=outer_its,
                    raise_on_error=False)
    return time.perf_counter() - t0, st, oracle.get_threads()


def oracle_estimate(w, M: int, J: int):
    """Oracle time-to-solution for J outer iterations from three bounded samples.

    Outer iteration j costs one RAS application plus a CGS2 against j+1 basis vectors, so past
    the first iterations (cheaper while the Krylov vectors still vanish on most subdomains) the
    cost per iteration grows linearly in j.  The solve is timed to M/4, M/2 and M iterations
    (separate runs, after an untimed 10-iteration warm-up of the oracle's threads); the mean
    costs per iteration over the windows [M/4, M/2) and [M/2, M) give that line, which is summed
    from M to J and added to t(M)."""
    oracle_sample(w, 10)
    t0, st0, cores = oracle_sample(w, max(1, M // 4))
    t1, st1, _ = oracle_sample(w, max(2, M // 2))
    t2, st2, _ = oracle_sample(w, M)
    j0, j1, j2 = st0["outer_its"], st1["outer_its"], st2["outer_its"]
    if j2 >= J or not (j0 < j1 < j2):
        return t2 * J / max(1, j2), cores, f"first {j2} of {J} outer iterations, scaled linearly"
    r1 = (t1 - t0) / (j1 - j0)                  # mean cost per iteration over [j0, j1)
    r2 = (t2 - t1) / (j2 - j1)                  # ... over [j1, j2)
    m1, m2 = (j0 + j1 + 1) / 2.0, (j1 + j2 + 1) / 2.0
    c = max(0.0, (r2 - r1) / (m2 - m1))         # growth per iteration (the CGS2 term)
    est = t2 + (J - j2) * r2 + c * ((J * (J + 1) - j2 * (j2 + 1)) / 2.0 - (J - j2) * m2)
    return est, cores, (f"first {j0}, {j1} and {j2} of {J} outer iterations timed ({t0:.2f} s, "
                        f"{t1:.2f} s, {t2:.2f} s); the cost per iteration, linear in j through "
                        f"the two later windows, summed to J={J}")


WARM_START_PARAMS = os.path.join(ROOT, "paper_2103_17081_gb300", "weights", "k200_warmstart.bin")


def oracle_error(w, x, name=None):
    """Relative error of the solution x (device tensor, one RHS) against the oracle's stored
    solve `name` (default: workload w's own): 2-norm and largest entry error over the largest
    entry; None when no stored solve exists."""
    import numpy as np
    name = name or w.name
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle_x.npy")
    if not os.path.exists(path) or w.nrhs != 1:
        return None
    xr = np.load(path)
    xg = x.detach().cpu().numpy()
    if xr.dtype.kind == "f":          # real data: the oracle stores Re x (its Im x is exactly 0)
        xr = xr.astype(np.complex128)
    d = xg - xr
    return {"rel_2norm": float(np.linalg.norm(d) / np.linalg.norm(xr)),
            "max_rel": float(np.max(np.abs(d)) / np.max(np.abs(xr))),
            "reference": f"tests/golden/{name}_oracle_x.npy (oracle, complex128)"}


def time_form(s, f, x, kw, steps, warmup, flush, stream):
    """Mean CUDA-event time of `steps` solves after `warmup` untimed ones (L2 flushed before each
    timed solve), with the stats of the last."""
    import torch
    for _ in range(warmup):
        s.solve(f, out=x, **kw)
    torch.cuda.synchronize()
    ts, st = [], None
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = s.solve(f, out=x, **kw)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.mean(ts), st


def apply_options(s, opts):
    """--option NAME=VALUE pairs: implementation choices of the solver (hdd_set_option)."""
    for o in opts:
        name, _, val = o.partition("=")
        s.set_option(name.strip(), int(val))


def workload_config(w) -> dict:
    """Keys that define the workload; both arms report them identically."""
    return {"workload": w.name, "k": w.k, "N": w.N, "ppwl": round(w.ppwl, 2),
            "subdomains": f"{w.Sx}x{w.Sy}", "overlap": w.overlap, "nrhs": w.nrhs,
            "inner_tol": w.inner_tol, "outer_tol": w.outer_tol,
            "boundary": "impedance" if w.bc else "dirichlet"}


def run_reference(args):
    """CPU oracle arm: each timed step times the oracle on bounded samples of the workload and
    extrapolates to the full outer count (oracle_estimate); an untimed warm-up step is a short
    10-iteration oracle solve (each estimate warms the oracle up again on its own)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = W.make(args.workload)
    J = args.full_outer_its
    for _ in range(args.warmup):
        oracle_sample(w, 10)
    times = []
    for _ in range(args.steps):
        est, cores, how = oracle_estimate(w, args.sample_its, J)
        times.append(est)
    v = statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": dict(workload_config(w), inner_prec=128, parallelism="single"),
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": "per step: " + how},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2103_17081_gb300 import Solver

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    w = W.make(args.workload, seed=rank)          # independent replica per rank
    s = Solver.from_workload(w, device=dev)
    apply_options(s, args.option)
    f = s.build_rhs_batch(w.rhs) if w.nrhs > 1 else s.build_rhs(w.rhs[0])
    x = s.empty(f.numel())
    kw = dict(outer_tol=w.outer_tol, inner_tol=w.inner_tol, inner_prec=args.prec,
              outer_restart=args.outer_maxit, outer_maxit=args.outer_maxit,
              outer_reorth32=0 if args.fp64_reorth else 1)
    tiles = None
    if args.autotune:
        tiles = s.autotune(inner_tol=w.inner_tol, inner_prec=args.prec)
    if args.warm_start:
        from paper_2103_17081_gb300 import warmstart
        s.cnn_set_params(warmstart.load(args.warm_start))
        kw["warm_start"] = 1
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    kw["raise_on_error"] = args.outer_maxit >= 2000   # a lowered limit is a bounded profiling run
    for _ in range(args.warmup):
        s.solve(f, out=x, **kw)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(dev)
    clocks.start()
    l0 = s.launch_count()
    times, stats = [], None
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)                                  # evict L2 between timed solves
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, stats = s.solve(f, out=x, **kw)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    barrier()
    launches = s.launch_count() - l0
    clk = clocks.stop()
    # kernel table and roofline: one more (untimed) solve with the per-launch CUDA-event profiler
    # on; the timed solves above run without it
    flush.fill_(1.0)
    s.profile(True)
    s.solve(f, out=x, **kw)
    prof = s.profile_stats()
    s.profile(False)
    t_step = statistics.mean(times)
    t_step = max_over_ranks(t_step, f"cuda:{dev}")

    # end to end: pinned host f → device, solve, device → host x, every step
    fh = f.cpu().pin_memory()
    xh = torch.empty_like(fh).pin_memory()
    fd = torch.empty_like(f)
    e2e = []
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fd.copy_(fh, non_blocking=True)
        s.solve(fd, out=x, **kw)
        xh.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)

    # check the answer on the device: true relative residual, and the error against the oracle
    r = f - s.apply_A(x)
    rel = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(f))
    err = oracle_error(w, x) if rank == 0 else None     # the stored solves use seed 0

    # the other forms of the method, fewer steps each: plain FP64 (complex128 inner, FP64
    # second CGS pass), the learned warm start (network trained by the library's own kernels) and
    # the two-level hybrid RAS with the grid coarse space H = 2h (Dirichlet problem only)
    forms = {}
    if ws == 1 and args.form_steps > 0 and not args.warm_start and args.prec == 64 and not args.fp64_reorth:
        cand = [("plain_fp64", dict(kw, inner_prec=128, outer_reorth32=0), None)]
        if w.name == "k200" and os.path.exists(WARM_START_PARAMS):
            cand.append(("warm_start", dict(kw, warm_start=1), WARM_START_PARAMS))
        if w.bc == 0 and w.N % 2 == 0:
            cand.append(("two_level", dict(kw, two_level=1), None))
        for name, fkw, params in cand:
            if params:
                from paper_2103_17081_gb300 import warmstart
                s.cnn_set_params(warmstart.load(params))
            if fkw.get("two_level"):
                s.setup_coarse_grid(2)
            t, fst = time_form(s, f, x, fkw, args.form_steps, 1, flush, stream)
            forms[name] = {"value": t, "unit": "s", "steps": args.form_steps, "warmup": 1,
                           "outer_its": fst["outer_its"], "inner_its_avg": round(fst["inner_its_avg"], 3),
                           "rel_res_true": fst["rel_res_true"], "err_vs_oracle": oracle_error(w, x),
                           "inner_prec": fkw["inner_prec"],
                           "outer": OUTER_DF if fkw["outer_reorth32"] else "cgs2-fp64",
                           "warm_start": bool(fkw.get("warm_start", 0))}
            if params:
                forms[name]["params"] = os.path.relpath(params, ROOT)
            if fkw.get("two_level"):
                # against the oracle's own two-level solve, and the coarse-grid kernels' share of
                # one more (profiled) solve
                forms[name]["err_vs_oracle_two_level"] = oracle_error(w, x, w.name + "tl")
                forms[name]["coarse_grid"] = "P1, H = 2h, lumped mass, DST solve in FP32"
                s.profile(True)
                s.solve(f, out=x, **fkw)
                torch.cuda.synchronize()
                fam = {d["name"]: d for d in s.profile_stats()}
                s.profile(False)
                tot = sum(d["ms"] for d in fam.values())
                cg = fam.get("two_level_grid_coarse", {"ms": 0.0, "launches": 0})
                forms[name]["grid_coarse_ms"] = round(cg["ms"], 3)
                forms[name]["grid_coarse_launches"] = cg["launches"]
                forms[name]["grid_coarse_share"] = round(cg["ms"] / tot, 4) if tot > 0 else None
        forms["default_faster_than_plain_fp64"] = t_step < forms["plain_fp64"]["value"]
        if "two_level" in forms:
            forms["two_level_faster_than_default"] = forms["two_level"]["value"] < t_step

    # roofline of the dominant kernel family (CUDA-event time inside the timed region)
    hbm, hbm_src = _peaks()
    dom = max(prof, key=lambda d: d["ms"])
    per_launch_ms = dom["ms"] / max(1, dom["launches"])
    fp64_frac = dom["flops"] / (dom["ms"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS
    hbm_frac = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9 / hbm
    # double-FP32 families count FP32 instructions as their work (12 per product of pairs)
    fp32_frac = dom["flops"] / (dom["ms"] * 1e-3) / 1e12 / FP32_PEAK_TINSTR
    if dom["bound"] == "fp64" and fp64_frac >= hbm_frac:      # the roof it sits closer to binds
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "kernel": dom["name"],
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (measured 1.19)",
                "hbm_frac": hbm_frac}
    elif dom["bound"] == "fp32" and fp32_frac >= hbm_frac:
        ach = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TINSTR, "unit": "T FP32 instructions/s",
                "frac": ach / FP32_PEAK_TINSTR, "traffic": None, "kernel": dom["name"],
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                "hbm_frac": hbm_frac}
    else:
        ach = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel": dom["name"], "peak_source": hbm_src,
                "fp64_frac": fp64_frac if dom["bound"] == "fp64" else None,
                "fp32_instr_frac": fp32_frac if dom["bound"] == "fp32" else None}
    roof["launches"] = dom["launches"]
    roof["ms_per_launch"] = per_launch_ms
    df = any(d["name"] == "outer_dots_df32" and d["launches"] for d in prof)
    ratio = TRAFFIC_PER_ALG.get((dom["name"], df))
    if ratio is not None and w.name == "k200" and w.nrhs == 1 and args.prec == 64 and not args.fp64_reorth:
        # the configuration of the ncu capture; elsewhere (bases that fit in L2, other kernels)
        # no measured traffic exists and the field stays null
        roof["traffic"] = dom["bytes"] / max(1, dom["launches"]) * ratio
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the family's kernels at "
                                  "outer iteration 200 (profiles/), scaled by basis vectors to this run's "
                                  "average launch")
    fams = {d["name"]: {"ms": round(d["ms"], 3), "launches": d["launches"],
                        "GB/s": round(d["bytes"] / max(d["ms"], 1e-9) / 1e6, 1),
                        "TFLOP/s": round(d["flops"] / max(d["ms"], 1e-9) / 1e9, 4)}
            for d in prof}
    local_fams = [d for d in prof if d["name"].startswith("local_")]
    lb = sum(d["bytes"] for d in local_fams)
    lt = sum(d["ms"] for d in local_fams)
    subdomain_gbs = lb / max(lt, 1e-9) / 1e6

    line = {"metric": METRIC, "value": t_step, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64-inner/f64-outer" if args.prec == 64 else "c128",
            "data": "synthetic",
            "config": {**workload_config(w), "inner_prec": args.prec,
                       "l2": "flushed between timed steps (512 MB write)",
                       "warm_start": bool(args.warm_start), "outer": "cgs2-fp64" if args.fp64_reorth else OUTER_DF,
                       "tiles": tiles or {"fine_rows": 8, "coarse_rows": 4},
                       "parallelism": "replicas" if ws > 1 else "single",
                       **({"options": list(args.option)} if args.option else {})},
            "solve": {"outer_its": stats["outer_its"], "inner_its_avg": round(stats["inner_its_avg"], 3),
                      "rel_res_true": rel, "status": stats["status_code"], "err_vs_oracle": err},
            "forms": forms,
            "subdomain_solve_GBps": subdomain_gbs, "subdomain_solve_frac_hbm": subdomain_gbs / hbm,
            "roofline": roof, "kernels": fams,
            "e2e": {"value": statistics.mean(e2e) if e2e else None, "unit": "s",
                    "h2d_bytes_per_step": int(f.numel() * 16),
                    "d2h_bytes_per_step": int(x.numel() * 16)},
            "gpu_launches": int(launches), "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        est, cores, how = oracle_estimate(w, args.sample_its, stats["outer_its"])
        line["cpu_baseline"] = {"value": est, "unit": "s", "cores": cores, "kind": "oracle",
                                "sample": how}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ras_dense(args):
    """Subdomain-solve throughput: `args.ras_dense` timed RAS applications (after one untimed) of a
    seeded dense vector, so every (subdomain, RHS) task is active, complex64 inner solves to the
    workload's tolerance; per kernel family the CUDA-event time, launches and algorithmic GB/s,
    and the subdomain-solve families (local_* and the coarse solve) against the HBM peak.  Prints
    one JSON line (not the time-to-solution line)."""
    import torch

    from paper_2103_17081_gb300 import Solver

    w = W.make(args.workload)
    s = Solver.from_workload(w)
    apply_options(s, args.option)
    if args.autotune:
        s.autotune(inner_tol=w.inner_tol, inner_prec=args.prec)
    n = s.n
    g = torch.Generator(device="cuda").manual_seed(5)
    v = torch.complex(torch.rand(s.nrhs * n, generator=g, device="cuda", dtype=torch.float64) - 0.5,
                      torch.rand(s.nrhs * n, generator=g, device="cuda", dtype=torch.float64) - 0.5)
    for r in range(s.nrhs):
        v[r * n:(r + 1) * n] /= torch.linalg.vector_norm(v[r * n:(r + 1) * n])
    z = s.empty(v.numel())
    kw = dict(inner_tol=w.inner_tol, inner_prec=args.prec)
    s.ras_apply(v, out=z, **kw)
    torch.cuda.synchronize()
    s.profile(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    its = []
    for _ in range(args.ras_dense):
        _, its = s.ras_apply(v, out=z, **kw)
    e1.record(stream)
    e1.synchronize()
    prof = s.profile_stats()
    s.profile(False)
    hbm, hbm_src = _peaks()
    fams = {d["name"]: {"ms": round(d["ms"], 3), "launches": d["launches"],
                        "GB/s": round(d["bytes"] / max(d["ms"], 1e-9) / 1e6, 1)}
            for d in prof if d["launches"]}
    loc = [d for d in prof if d["name"].startswith("local_")]
    sub = loc + [d for d in prof if d["name"] == "coarse_solve_fp64"]
    lgbs = sum(d["bytes"] for d in loc) / max(sum(d["ms"] for d in loc), 1e-9) / 1e6
    print(json.dumps({"mode": "ras_dense", "config": workload_config(w), "inner_prec": args.prec,
                      "applications": args.ras_dense, "ms_per_application": e0.elapsed_time(e1) / args.ras_dense,
                      "inner_its_avg": sum(its) / max(1, len(its)), "inner_its_max": max(its) if its else 0,
                      "local_GBps": lgbs, "local_frac_hbm": lgbs / hbm,
                      "local_ms": sum(d["ms"] for d in loc), "subdomain_ms": sum(d["ms"] for d in sub),
                      "hbm_peak": hbm, "peak_source": hbm_src, "kernels": fams}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="k200")
    ap.add_argument("--prec", type=int, default=64, choices=[64, 128])
    ap.add_argument("--outer-maxit", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--sample-its", type=int, default=400)
    ap.add_argument("--full-outer-its", type=int, default=0)
    ap.add_argument("--option", action="append", default=[],
                    help="NAME=VALUE: a hdd_set_option choice of the solver (Solver.OPTIONS), repeatable")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form-steps", type=int, default=2,
                    help="timed solves of each other form (plain FP64, warm start); 0 skips them")
    ap.add_argument("--warm-start", default=None,
                    help="parameter file of a trained warm-start network (written by "
                         "python -m paper_2103_17081_gb300.warmstart train)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the local tile shapes with hdd_autotune before the warm-up")
    ap.add_argument("--fp64-reorth", action="store_true",
                    help="second outer CGS pass in FP64 (default: guarded FP32 correction)")
    ap.add_argument("--ras-dense", type=int, default=0,
                    help="instead of solves: time this many RAS applications of a dense seeded vector "
                         "(every local solve active) and report the subdomain-solve kernels' bandwidth")
    args = ap.parse_args()
    if args.ras_dense > 0:
        return run_ras_dense(args)
    if args.impl == "reference":
        if not args.full_outer_its:
            args.full_outer_its = {"tiny": 18, "k100": 282, "k200": 1270, "k200s": 781}.get(args.workload, 1270)
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
