"""Write tests/golden/k200_oracle.json: the CPU oracle's solve of the k=200 workload.

Runs only oracle/ (no CUDA code).  Stores the outer/inner iteration counts, the residual history
every 50 iterations, ||x||_2, ||x||_inf and the solution at 256 seeded interior nodes, which the
GPU test compares against at full size.  Takes ~20 minutes on 8 cores.

    python tests/golden/make_k200_reference.py
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


def main():
    w = W.make("k200")
    p = oracle.from_workload(w)
    f = p.rhs(w.rhs[0])
    t0 = time.time()
    x, st = p.solve(f, outer_tol=w.outer_tol, inner_tol=w.inner_tol)
    rng = W.SplitMix64(2024)
    idx = sorted({int(rng.uniform(0, p.n)) for _ in range(256)})
    out = {
        "workload": w.name, "N": w.N, "k": w.k, "outer_tol": w.outer_tol, "inner_tol": w.inner_tol,
        "outer_restart": 2000, "inner_restart": 30,
        "outer_its": st["outer_its"], "inner_its_total": st["inner_its_total"],
        "inner_its_avg": st["inner_its_avg"], "rel_res_true": st["rel_res_true"],
        "res_history_every_50": [float(v) for v in st["res_history"][::50]],
        "x_norm2": float(np.linalg.norm(x)), "x_norminf": float(np.max(np.abs(x))),
        "x_imag_max": float(np.max(np.abs(x.imag))),
        "sample_index": idx, "sample_re": [float(x[i].real) for i in idx],
        "oracle_seconds": time.time() - t0, "oracle_threads": oracle.get_threads(),
    }
    with open(os.path.join(HERE, "k200_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not k.startswith("sample")}))


if __name__ == "__main__":
    main()
