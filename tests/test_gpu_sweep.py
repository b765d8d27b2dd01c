"""The paper's iteration-count study (§3, Tables 1–4) and the k=100 inner-tolerance sweep on the
GPU, against the CPU oracle, through the C ABI.

1. A few cells of the paper's settings (h = 1/n_glob with n_glob = 1.5k, one element layer of
   overlap, N = S² square subdomains, a centred point source, outer FGMRES to 1e-6) run by
   paper_2103_17081_gb300.sweep with complex128 inner solves: the GPU's outer iteration count and
   average inner count per subdomain solve must equal the oracle's (outer ±1, or ±10 % where the
   oracle's residual history stagnates within 4x of the tolerance at the earlier stopping point;
   at inner tolerance 1e-10 both sides take the same stopping decisions).  The paper's own counts (FreeFem/PETSc,
   other restart and partition-of-unity settings) are printed beside them as context: they are
   trends, not values to reproduce.
2. The k=100 workload (N=320, 4x4 subdomains, overlap 2, point source + seeded bump) with inner
   tolerances {1e-1, 1e-2, 1e-4, exact}, the plain FP64 form (complex128 inner, FP64 outer),
   against the oracle's solves stored by tests/golden/make_k100_sweep_reference.py: outer
   iterations ±1, the solution within 1e-5 of the oracle's (normwise and at every node, relative
   to max|x|).
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# The paper's cells "outer (average inner)" at 10 points per wavelength: Table 1 (LU, outer only)
# and Table 2 (inner 1e-10), k = 20 and 40, N = 4 and 9 subdomains.
PAPER = {("LU", 20, 4): (20, None), ("LU", 20, 9): (27, None), ("LU", 40, 4): (31, None),
         ("LU", 40, 9): (60, None), ("1e-10", 20, 4): (20, 23), ("1e-10", 20, 9): (27, 25),
         ("1e-10", 40, 4): (32, 35), ("1e-10", 40, 9): (62, 29)}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def test_paper_table_cells_match_oracle(oracle_mod):
    _torch()
    from paper_2103_17081_gb300 import sweep
    tols = [("LU", 0.0), ("1e-10", 1e-10)]
    rows = sweep.run([20, 40], [10], tols, [2, 3], inner_prec=128, log=None)
    assert len(rows) == 8
    setting = {(k, S): w for (_, k, _, S, w) in sweep.settings([20, 40], [10], [2, 3])}
    lines = []
    for r in rows:
        S = int(round(r["N"] ** 0.5))
        w = setting[(r["k"], S)]
        tol = dict(tols)[r["inner"]]
        p = oracle_mod.from_workload(w, exact=tol <= 0)
        _, so = p.solve(p.rhs(w.rhs[0]), outer_tol=1e-6, inner_tol=tol)
        assert r["status"] == 0 and r["rel_res"] <= 1.0001e-6
        d = abs(r["outer_its"] - so["outer_its"])
        if d > 1:
            # a stagnation plateau at the tolerance: the oracle's residual at the earlier of the
            # two stopping points is already within 4x of it, so rounding-level differences in
            # the preconditioner (1e-14 here; histories equal to 1e-7 through iteration 24 at
            # k=20, N=9) move the stopping point by a few iterations
            ho = so["res_history"]
            i = min(r["outer_its"], so["outer_its"]) - 1
            assert ho[i] <= 4e-6 and d <= max(2, 0.1 * so["outer_its"]), (r, so["outer_its"], ho[i])
        if tol > 0:
            assert abs(r["inner_avg"] - round(so["inner_its_avg"], 1)) <= 0.15, (r, so["inner_its_avg"])
        po, pi = PAPER[(r["inner"], r["k"], r["N"])]
        lines.append(f"inner {r['inner']:>5} k={r['k']:>3} N={r['N']:>2}: gpu {r['outer_its']} "
                     f"({r['inner_avg']}), oracle {so['outer_its']} ({so['inner_its_avg']:.1f}), "
                     f"paper {po}" + (f" ({pi})" if pi else ""))
    print("\n" + "\n".join(lines))
    # the paper's trend: more outer iterations at the higher wavenumber, for each N and inner solve
    for name, _ in tols:
        for N in (4, 9):
            o = {r["k"]: r["outer_its"] for r in rows if r["inner"] == name and r["N"] == N}
            assert o[40] > o[20]


def test_k100_inner_tolerance_sweep_matches_stored_oracle():
    torch = _torch()
    from paper_2103_17081_gb300 import Solver, sweep
    ref = json.load(open(os.path.join(GOLD, "k100_sweep_oracle.json")))
    xs = np.load(os.path.join(GOLD, "k100_sweep_oracle_x.npz"))
    w = W.make("k100")
    s = Solver.from_workload(w, exact=True)
    f = s.build_rhs(w.rhs[0])
    rows = sweep.c2_sweep(s, f, log=None)
    assert [r["inner"] for r in rows] == [c["inner"] for c in ref["cases"]]
    for r, c in zip(rows, ref["cases"]):
        x = r.pop("x")
        assert r["status"] == 0
        assert float(torch.linalg.vector_norm(f - s.apply_A(x)) / torch.linalg.vector_norm(f)) <= 1.0001e-6
        assert abs(r["outer_its"] - c["outer_its"]) <= 1, (r, c)
        xg = x.cpu().numpy()
        assert float(np.max(np.abs(xg.imag))) == 0.0
        xr = xs[c["inner"]]
        err2 = np.linalg.norm(xg.real - xr) / np.linalg.norm(xr)
        errm = float(np.max(np.abs(xg.real - xr))) / float(np.max(np.abs(xr)))
        assert err2 < 1e-5 and errm < 1e-5, (c["inner"], err2, errm)
