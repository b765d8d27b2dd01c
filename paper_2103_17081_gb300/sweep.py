"""The settings of the paper's iteration-count study (§3, Tables 1–4) run on the GPU.

Every row: wavenumber k ∈ {20, 40, 80, 160} at about 10 or 20 points per wavelength with
h = 1/n_glob (n_glob = 1.5k or 3k intervals per side), N = 4, 9, 16 or 25 square subdomains with
one element layer of overlap, a unit point source at the centre, outer FGMRES to relative
residual 1e-6, and subdomain solves by banded LU (Table 1) or by deflated GMRES to 1e-10, 1e-5 or
1e-2 (Tables 2–4).  Each entry is "outer (average inner)" as in the paper's tables, the average
being the inner iterations per subdomain solve.  The paper's own numbers come from FreeFem/PETSc
with an unstated restart length and partition of unity, so they are trends to compare with, not
values to reproduce.

--c2 runs the k=100 workload instead (N=320, 4x4 subdomains, overlap 2, centre point source plus
a seeded Gaussian bump) with inner tolerances 1e-1, 1e-2, 1e-4 and exact (banded LU) subdomain
solves in the plain FP64 form (complex128 inner, FP64 outer), timing each solve.

With --bc 1 the same settings run with the impedance (Sommerfeld) condition du/dn - iku = 0 on
all four sides instead of u = 0; the paper states the solver suits that problem (§3) but prints
no iteration counts for it.

    python -m paper_2103_17081_gb300.sweep [--ppwl 10 20] [--k 20 40 80 160] [--bc 0|1] [--json out.jsonl]
    python -m paper_2103_17081_gb300.sweep --c2
"""
from __future__ import annotations

import argparse
import json
import time

TOLS = [("LU", 0.0), ("1e-10", 1e-10), ("1e-5", 1e-5), ("1e-2", 1e-2)]
SUBS = [2, 3, 4, 5]                      # N = S² subdomains


def settings(ks, ppwls, subs, bc=0):
    """(ppwl, k, n_glob, S, workload) of every setting: h = 1/n_glob with n_glob = 1.5k (10 ppwl)
    or 3k (20 ppwl), S x S subdomains, one element layer of overlap, centred point source."""
    import workloads as W
    out = []
    for ppwl in ppwls:
        for k in ks:
            n_glob = int(round(k * (1.5 if ppwl == 10 else 3.0)))
            for S in subs:
                out.append((ppwl, k, n_glob, S,
                            W.custom(float(k), n_glob, S, 1, name=f"k{k}_n{n_glob}_S{S}", bc=bc)))
    return out


def run(ks, ppwls, tols, subs, inner_prec=128, log=print, bc=0, two_level=0):
    """One solve per (setting, inner tolerance).  With complex128 inner solves the outer Arnoldi
    runs in plain FP64 as well (the form whose counts follow the oracle's stopping decisions);
    with complex64 ones it uses the default double-FP32 dots and guarded FP32 second pass.
    two_level: the hybrid two-level RAS with the grid coarse space H = 2h."""
    import torch

    from .solver import Solver

    rows = []
    for (ppwl, k, n_glob, S, w) in settings(ks, ppwls, subs, bc):
        need_lu = any(t <= 0 for _, t in tols)
        s = Solver.from_workload(w, exact=need_lu)
        if two_level:
            s.setup_coarse_grid(2)
        f = s.build_rhs(w.rhs[0])
        for name, tol in tols:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = s.solve(f, outer_tol=1e-6, inner_tol=tol, inner_prec=inner_prec,
                            inner_restart=30, inner_maxit=1000, raise_on_error=False,
                            outer_reorth32=int(inner_prec == 64), two_level=two_level)
            torch.cuda.synchronize()
            r = {"ppwl": ppwl, "k": k, "n_glob": n_glob, "N": S * S, "inner": name,
                 "outer_its": st["outer_its"], "inner_avg": round(st["inner_its_avg"], 1),
                 "rel_res": st["rel_res_true"], "status": st["status_code"],
                 "s": round(time.perf_counter() - t0, 3), "bc": bc, "two_level": int(bool(two_level))}
            rows.append(r)
            if log:
                log(json.dumps(r))
        del s
    return rows


C2_TOLS = [("1e-1", 1e-1), ("1e-2", 1e-2), ("1e-4", 1e-4), ("LU", 0.0)]


def c2_sweep(solver, f, log=print, reps: int = 1):
    """Inner-tolerance sweep of one solver (set up with exact local factors as well): each
    setting of C2_TOLS solved in the plain FP64 form, after one untimed warm-up solve, timed with
    CUDA events on the current stream (mean of `reps`).  Rows carry the last solution as "x"."""
    import torch

    rows = []
    for name, tol in C2_TOLS:
        kw = dict(outer_tol=1e-6, inner_tol=tol, inner_prec=128, outer_reorth32=0, raise_on_error=False)
        x, st = solver.solve(f, **kw)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x, st = solver.solve(f, out=x, **kw)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        r = {"inner": name, "outer_its": st["outer_its"], "inner_avg": round(st["inner_its_avg"], 2),
             "rel_res": st["rel_res_true"], "status": st["status_code"], "s": round(sum(ts) / len(ts), 4),
             "x": x}
        rows.append(r)
        if log:
            log(json.dumps({k: v for k, v in r.items() if k != "x"}))
    return rows


def table(rows, inner):
    """Markdown table of one inner setting, rows (ppwl, k), columns N."""
    sel = [r for r in rows if r["inner"] == inner]
    Ns = sorted({r["N"] for r in sel})
    out = ["| ppwl | k | n_glob | " + " | ".join(f"N={n}" for n in Ns) + " |",
           "|---|---|---|" + "---|" * len(Ns)]
    for ppwl in sorted({r["ppwl"] for r in sel}):
        for k in sorted({r["k"] for r in sel}):
            cells, ng = [], ""
            for n in Ns:
                m = [r for r in sel if r["ppwl"] == ppwl and r["k"] == k and r["N"] == n]
                if not m:
                    cells.append("")
                    continue
                r = m[0]
                ng = r["n_glob"]
                cells.append(str(r["outer_its"]) if inner == "LU" else f"{r['outer_its']} ({r['inner_avg']:g})")
            out.append(f"| {ppwl} | {k} | {ng} | " + " | ".join(cells) + " |")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2103_17081_gb300.sweep")
    ap.add_argument("--ppwl", type=int, nargs="+", default=[10, 20], choices=[10, 20])
    ap.add_argument("--k", type=int, nargs="+", default=[20, 40, 80, 160])
    ap.add_argument("--inner", nargs="+", default=[n for n, _ in TOLS], choices=[n for n, _ in TOLS])
    ap.add_argument("--subdomains", type=int, nargs="+", default=SUBS, help="S for S x S subdomains")
    ap.add_argument("--prec", type=int, default=128, choices=[64, 128], help="inner precision")
    ap.add_argument("--bc", type=int, default=0, choices=[0, 1],
                    help="0: u = 0 on the boundary (the paper's tables); 1: impedance condition")
    ap.add_argument("--two-level", action="store_true",
                    help="hybrid two-level RAS with the grid coarse space H = 2h (bc 0 only)")
    ap.add_argument("--json", default=None, help="also write every row as a JSON line to this file")
    ap.add_argument("--c2", action="store_true",
                    help="the k=100 inner-tolerance sweep {1e-1, 1e-2, 1e-4, exact} instead")
    ap.add_argument("--reps", type=int, default=3, help="timed solves per setting of --c2")
    a = ap.parse_args(argv)
    if a.c2:
        import workloads as W

        from .solver import Solver
        w = W.make("k100")
        s = Solver.from_workload(w, exact=True)
        c2_sweep(s, s.build_rhs(w.rhs[0]), reps=a.reps)
        return 0
    tols = [(n, t) for n, t in TOLS if n in a.inner]
    rows = run(a.k, a.ppwl, tols, a.subdomains, a.prec, bc=a.bc, two_level=int(a.two_level))
    if a.json:
        with open(a.json, "w") as fh:
            for r in rows:
                fh.write(json.dumps(r) + "\n")
    for name, _ in tols:
        print(f"\ninner {name}:\n" + table(rows, name))
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
