"""Write tests/golden/k100_sweep_oracle.json and k100_sweep_oracle_x.npz: the CPU oracle's solves
of the k=100 workload (N=320, 4x4 subdomains, overlap 2, centre point source plus seeded
Gaussian bump, outer FGMRES to 1e-6) with inner deflated GMRES to 1e-1, 1e-2, 1e-4 and with
exact (banded LU) subdomain solves.

Runs only oracle/ (no CUDA code).  The .json holds the iteration counts and residuals, the .npz
the whole solution of each setting as float64 Re x (Im x is exactly zero for real data, which
the script asserts).  A few minutes on 8 cores.

    python tests/golden/make_k100_sweep_reference.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402

TOLS = [("1e-1", 1e-1), ("1e-2", 1e-2), ("1e-4", 1e-4), ("LU", 0.0)]


def main():
    w = W.make("k100")
    p = oracle.from_workload(w, exact=True)
    f = p.rhs(w.rhs[0])
    cases, xs = [], {}
    for name, tol in TOLS:
        t0 = time.time()
        x, st = p.solve(f, outer_tol=w.outer_tol, inner_tol=tol)
        assert float(np.max(np.abs(x.imag))) == 0.0
        xs[name] = np.ascontiguousarray(x.real)
        cases.append({"inner": name, "inner_tol": tol, "outer_its": st["outer_its"],
                      "inner_its_total": st["inner_its_total"], "inner_its_avg": st["inner_its_avg"],
                      "rel_res_true": st["rel_res_true"], "x_norm2": float(np.linalg.norm(x)),
                      "oracle_seconds": time.time() - t0})
        print(json.dumps(cases[-1]), flush=True)
    out = {"workload": w.name, "N": w.N, "k": w.k, "outer_tol": w.outer_tol, "outer_restart": 2000,
           "inner_restart": 30, "oracle_threads": oracle.get_threads(), "cases": cases,
           "solution_file": "k100_sweep_oracle_x.npz"}
    np.savez_compressed(os.path.join(HERE, "k100_sweep_oracle_x.npz"), **xs)
    with open(os.path.join(HERE, "k100_sweep_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
