"""Write the CPU oracle's solve of a k=200 workload under tests/golden/.

Runs only oracle/ (no CUDA code).  For workload W (k200: Dirichlet, the default; k200s: the
impedance boundary; k200tl: k200 with the two-level hybrid RAS preconditioner, grid coarse
space H = 2h) it writes

  W_oracle.json   outer/inner iteration counts, the residual history every 50 iterations,
                  ||x||_2, ||x||_inf and x at 256 seeded nodes;
  W_oracle_x.npy  the whole solution: float64 Re x for k200 (Im x is exactly 0 for real data,
                  which the script asserts), complex128 x for k200s.

The GPU tests compare their full-size solves against these at every node.  Each solve takes
10-25 minutes on 8 cores.

    python tests/golden/make_k200_reference.py [k200|k200s|k200tl]
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


def main(name: str = "k200"):
    two_level = name.endswith("tl")
    w = W.make(name[:-2] if two_level else name)
    p = oracle.from_workload(w)
    if two_level:
        p.setup_coarse_grid(2)
    f = p.rhs(w.rhs[0])
    t0 = time.time()
    x, st = p.solve(f, outer_tol=w.outer_tol, inner_tol=w.inner_tol, two_level=int(two_level))
    secs = time.time() - t0
    rng = W.SplitMix64(2024)
    idx = sorted({int(rng.uniform(0, p.n)) for _ in range(256)})
    out = {
        "workload": w.name, "two_level": int(two_level), "coarse_factor": 2 if two_level else 0, "N": w.N, "k": w.k, "bc": w.bc, "outer_tol": w.outer_tol,
        "inner_tol": w.inner_tol, "outer_restart": 2000, "inner_restart": 30,
        "outer_its": st["outer_its"], "inner_its_total": st["inner_its_total"],
        "inner_its_avg": st["inner_its_avg"], "rel_res_true": st["rel_res_true"],
        "res_history_every_50": [float(v) for v in st["res_history"][::50]],
        "x_norm2": float(np.linalg.norm(x)), "x_norminf": float(np.max(np.abs(x))),
        "x_imag_max": float(np.max(np.abs(x.imag))),
        "sample_index": idx, "sample_re": [float(x[i].real) for i in idx],
        "sample_im": [float(x[i].imag) for i in idx],
        "oracle_seconds": secs, "oracle_threads": oracle.get_threads(),
        "solution_file": f"{name}_oracle_x.npy",
    }
    if w.bc == 0:
        # real data and a real operator: the oracle keeps Im x exactly zero, so Re x is all of x
        assert out["x_imag_max"] == 0.0
        np.save(os.path.join(HERE, f"{name}_oracle_x.npy"), np.ascontiguousarray(x.real))
    else:
        np.save(os.path.join(HERE, f"{name}_oracle_x.npy"), np.ascontiguousarray(x))
    with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not k.startswith("sample")}))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "k200")
