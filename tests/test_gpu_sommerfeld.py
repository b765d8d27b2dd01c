"""GPU parity of the impedance (Sommerfeld) variant against the CPU oracle, through the C ABI.

The variant: du/dn - i k u = 0 on all four sides, every mesh node an unknown, A complex
symmetric; E and A_j are factored on the device as their real equivalents (the oracle factors
them as complex band matrices, so pivots differ and only rounding separates the two).  Bars, as
for the Dirichlet problem: load vector, global stencil and restriction to rounding (1e-14, the
restriction exactly); complex128 local operators to 1e-13 (P A, whose rounding the local
deflated conditioning amplifies, to 1e-11; coarse and direct solves to 1e-11 and 1e-10);
complex64 to FP32 rounding (2e-6, P A 1e-4); whole solves reach the outer tolerance on the
oracle's own matrix and match its solution to 1e-6 (complex128 inner) or 1e-5 (complex64
inner) relative, outer iteration counts within 10 % + 1.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def _to_dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _maxrel(a, b):
    """Largest entrywise error relative to the largest entry of b (a bar on every node)."""
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _close(a, b, tol):
    """Normwise and entrywise (relative to max|b|) agreement within tol."""
    return _rel(a, b) < tol and _maxrel(a, b) < tol


def _pair(oracle_mod, w, exact=False):
    from paper_2103_17081_gb300 import Solver
    _torch()
    s = Solver.from_workload(w, exact=exact)
    p = oracle_mod.from_workload(w, exact=exact)
    return s, p


# boxes touching one, two (corners) or no sides; uneven widths; overlap 1 and 2
CASES = [W.custom(13.0, 37, 3, 1, Sy=2, name="imp_ragged1", bc=1),
         W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45], name="imp_ragged2", bc=1),
         W.custom(20.0, 32, 2, 2, name="imp_k20", bc=1)]


@pytest.mark.parametrize("diag", [0, 1])
def test_rhs_and_global_operator(oracle_mod, diag):
    from paper_2103_17081_gb300 import Solver
    _torch()
    spec = W.RHSSpec([W.PointSource(0.0, 0.3), W.PointSource(1.0, 1.0, 2.0), W.PointSource(0.5, 0.5)],
                     [W.Bump(0.05, 0.9, 0.1, 1.5), W.Bump(0.6, 0.4, 0.07)])
    for (k, N) in [(13.0, 37), (20.0, 32)]:
        s = Solver(0).assemble(k, N, diag=diag, bc=1)
        p = oracle_mod.Problem(N, k, diag=diag, bc=1)
        assert s.n == p.n == (N + 1) ** 2
        assert _rel(s.build_rhs(spec).cpu().numpy(), p.rhs(spec)) < 1e-14
        x = W.random_complex_fast(p.n, 3)
        assert _rel(s.apply_A(_to_dev(x)).cpu().numpy(), p.apply(x)) < 1e-14


def test_boxes_and_ownership_match_oracle(oracle_mod):
    from paper_2103_17081_gb300 import Solver
    _torch()
    for w in CASES:
        s = Solver(0).assemble(w.k, w.N, bc=1).setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
        p = oracle_mod.Problem(w.N, w.k, bc=1)
        p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
        for q in range(p.nsub):
            g, o = s.subdomain(q), p.box(q)
            for key in ("ix0", "ix1", "iy0", "iy1", "ox0", "ox1", "oy0", "oy1", "nx", "ny"):
                assert g[key] == o[key], (w.name, q, key)


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
@pytest.mark.parametrize("prec", [128, 64])
def test_local_operators(oracle_mod, w, prec):
    s, p = _pair(oracle_mod, w, exact=True)
    fo, co = s.offsets()
    tol = 1e-13 if prec == 128 else 2e-6
    xf = W.random_complex_fast(fo[-1], 5)
    xc = W.random_complex_fast(co[-1], 6)
    xg = W.random_complex_fast(p.n, 7)
    if prec == 64:        # the complex64 path rounds inputs to FP32 first
        xf = xf.astype(np.complex64).astype(np.complex128)
        xc = xc.astype(np.complex64).astype(np.complex128)
        xg = xg.astype(np.complex64).astype(np.complex128)
    outs = {op: s.local_op(op, _to_dev(x), prec).cpu().numpy()
            for op, x in [("A", xf), ("Z", xc), ("Zt", xf), ("R", xg), ("PA", xf)]}
    if prec == 128:
        outs["Einv"] = s.local_op("Einv", _to_dev(xc)).cpu().numpy()
        outs["Ainv"] = s.local_op("Ainv", _to_dev(xf)).cpu().numpy()
    for q in range(p.nsub):
        F, Cc = slice(fo[q], fo[q + 1]), slice(co[q], co[q + 1])
        assert _rel(outs["A"][F], p.sub_apply_A(q, xf[F])) < tol
        assert _rel(outs["Z"][F], p.sub_apply_Z(q, xc[Cc])) < tol
        assert _rel(outs["Zt"][Cc], p.sub_apply_Zt(q, xf[F])) < tol
        assert _rel(outs["R"][F], p.restrict(q, xg)) == 0.0 or prec == 64
        if prec == 128:
            assert _rel(outs["PA"][F], p.sub_apply_PA(q, xf[F])) < 1e-11
        else:
            assert _close(outs["PA"][F], p.sub_apply_PA(q, xf[F]), 1e-4)
        if prec == 128:
            assert _rel(outs["Einv"][Cc], p.coarse_solve(q, xc[Cc])) < 1e-11
            assert _rel(outs["Ainv"][F], p.sub_solve_exact(q, xf[F])) < 1e-10


@pytest.mark.parametrize("prec,tol", [(128, 1e-6), (128, 1e-2), (64, 1e-2)])
def test_ras_apply_matches_oracle(oracle_mod, prec, tol):
    w = CASES[1]
    s, p = _pair(oracle_mod, w)
    v = W.random_complex_fast(p.n, 11)
    v /= np.linalg.norm(v)
    zg, its = s.ras_apply(_to_dev(v), inner_tol=tol, inner_prec=prec)
    zo, sto = p.ras_apply(v, tol)
    zg = zg.cpu().numpy()
    if prec == 128:
        assert sum(its) == sto["inner_its_total"]
        assert _rel(zg, zo) < 1e-9
    else:
        assert abs(sum(its) - sto["inner_its_total"]) <= max(2, 0.1 * sto["inner_its_total"])
        assert _close(zg, zo, 1e-4)


@pytest.mark.parametrize("prec", [128, 64])
def test_solve_matches_oracle(oracle_mod, prec):
    """k = 20, N = 32, 2x2 subdomains, overlap 2, centred point source, inner tolerance 1e-2."""
    w = CASES[2]
    s, p = _pair(oracle_mod, w)
    f = p.rhs(w.rhs[0])
    xo, sto = p.solve(f, outer_tol=1e-6, inner_tol=1e-2)
    xg, stg = s.solve(s.build_rhs(w.rhs[0]), outer_tol=1e-6, inner_tol=1e-2, inner_prec=prec)
    xg = xg.cpu().numpy()
    A = p.matrix("A")
    assert np.linalg.norm(f - A @ xg) <= 1e-6 * np.linalg.norm(f) * 1.0001
    assert _close(xg, xo, 1e-6 if prec == 128 else 1e-5)
    assert abs(stg["outer_its"] - sto["outer_its"]) <= 0.1 * sto["outer_its"] + 1
    assert np.linalg.norm(xg.imag) > 0.1 * np.linalg.norm(xg)        # a radiating solution


def test_exact_inner_solve_matches_oracle(oracle_mod):
    w = CASES[0]
    s, p = _pair(oracle_mod, w, exact=True)
    f = p.rhs(w.rhs[0])
    xo, sto = p.solve(f, outer_tol=1e-8, inner_tol=0.0)
    xg, stg = s.solve(s.build_rhs(w.rhs[0]), outer_tol=1e-8, inner_tol=0.0)
    assert stg["outer_its"] == sto["outer_its"]
    assert _rel(xg.cpu().numpy(), xo) < 1e-9


def test_k60_solve_matches_oracle(oracle_mod):
    """k = 60, N = 96 (about 10 points per wavelength), 3x3 subdomains, overlap 2, complex64
    inner solves to 1e-2: every box kind (corner, side, interior) in one solve."""
    w = W.custom(60.0, 96, 3, 2, name="imp_k60", bc=1)
    s, p = _pair(oracle_mod, w)
    f = p.rhs(w.rhs[0])
    xo, sto = p.solve(f, outer_tol=1e-6, inner_tol=1e-2)
    xg, stg = s.solve(s.build_rhs(w.rhs[0]), outer_tol=1e-6, inner_tol=1e-2, inner_prec=64)
    xg = xg.cpu().numpy()
    assert np.linalg.norm(f - p.matrix("A") @ xg) <= 1e-6 * np.linalg.norm(f) * 1.0001
    assert _close(xg, xo, 1e-5)
    assert abs(stg["outer_its"] - sto["outer_its"]) <= 0.1 * sto["outer_its"] + 1


def test_warm_start_is_refused_for_impedance():
    from paper_2103_17081_gb300 import Solver
    _torch()
    w = CASES[2]
    s = Solver.from_workload(w)
    with pytest.raises(Exception):
        s.cnn_set_params(np.zeros(s.cnn_num_params(), dtype=np.float32))


def test_k100_solve_matches_oracle(oracle_mod):
    """The k = 100 geometry (N = 320, 4x4 subdomains, overlap 2, 20 points per wavelength) with
    the impedance condition: complex64 inner solves to 1e-2, outer FGMRES to 1e-6."""
    w = W.custom(100.0, 320, 4, 2, name="imp_k100", bc=1)
    s, p = _pair(oracle_mod, w)
    f = p.rhs(w.rhs[0])
    xo, sto = p.solve(f, outer_tol=1e-6, inner_tol=1e-2)
    xg, stg = s.solve(s.build_rhs(w.rhs[0]), outer_tol=1e-6, inner_tol=1e-2, inner_prec=64)
    xg = xg.cpu().numpy()
    assert np.linalg.norm(f - p.matrix("A") @ xg) <= 1e-6 * np.linalg.norm(f) * 1.0001
    assert _close(xg, xo, 1e-5)
    assert abs(stg["outer_its"] - sto["outer_its"]) <= 0.1 * sto["outer_its"] + 1


def test_batched_rhs_match_single_rhs_runs(oracle_mod):
    """Three right-hand sides (one of them on the boundary of the square) in one batch give the
    per-RHS results of separate runs, and each matches the oracle."""
    from paper_2103_17081_gb300 import Solver
    torch = _torch()
    w = CASES[1]
    specs = [W.RHSSpec([W.PointSource(0.31, 0.62)]), W.RHSSpec([W.PointSource(1.0, 0.4)]),
             W.RHSSpec([W.PointSource(0.7, 0.2)], [W.Bump(0.5, 0.5, 0.1)])]
    s1 = Solver.from_workload(w)
    sb = Solver.from_workload(w).setup_batch(3)
    fb = sb.build_rhs_batch(specs)
    n = sb.n
    zb, itb = sb.ras_apply(fb / torch.linalg.vector_norm(fb), inner_tol=1e-2, inner_prec=64)
    xb, stb = sb.solve(fb, inner_prec=64)
    p = oracle_mod.from_workload(w)
    for r, spec in enumerate(specs):
        fr = fb[r * n:(r + 1) * n].clone()
        z1, it1 = s1.ras_apply(fr / torch.linalg.vector_norm(fb), inner_tol=1e-2, inner_prec=64)
        assert _rel(zb[r * n:(r + 1) * n].cpu().numpy(), z1.cpu().numpy()) <= 1e-14
        assert itb[r * s1.nsub:(r + 1) * s1.nsub] == it1
        x1, st1 = s1.solve(fr, inner_prec=64)
        assert _rel(xb[r * n:(r + 1) * n].cpu().numpy(), x1.cpu().numpy()) <= 1e-12
        xo, so = p.solve(p.rhs(spec))
        assert _close(xb[r * n:(r + 1) * n].cpu().numpy(), xo, 1e-5)
    assert stb["rel_res_true"] <= 1e-6 * 1.0001


def test_k200s_full_solve_against_stored_oracle():
    """The k=200 impedance workload (N=640, (N+1)² = 410,881 unknowns, 8x8 subdomains, the k200
    load), complex64 inner solves to 1e-2, outer FGMRES to 1e-6, against the oracle's solution
    stored by tests/golden/make_k200_reference.py (complex128): every node within 1e-5 of max|x|,
    the whole vector within 1e-5 relative in the 2-norm, outer iterations within +10 %."""
    import json
    import os
    torch = _torch()
    from paper_2103_17081_gb300 import Solver
    gold = os.path.join(os.path.dirname(__file__), "golden")
    ref = json.load(open(os.path.join(gold, "k200s_oracle.json")))
    xr = np.load(os.path.join(gold, "k200s_oracle_x.npy"))
    w = W.make("k200s")
    assert xr.shape == ((w.N + 1) ** 2,)
    s = Solver.from_workload(w)
    f = s.build_rhs(w.rhs[0])
    x, st = s.solve(f, outer_tol=w.outer_tol, inner_tol=w.inner_tol, inner_prec=64)
    r = f - s.apply_A(x)
    assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(f)) <= 1.0001e-6
    assert st["outer_its"] <= 1.1 * ref["outer_its"]
    xg = x.cpu().numpy()
    assert _close(xg, xr, 1e-5), (_rel(xg, xr), _maxrel(xg, xr))
