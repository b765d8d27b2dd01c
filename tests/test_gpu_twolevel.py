"""Two-level RAS with the grid coarse space (the conclusions, §4, name a coarse space as the next
step) on the GPU, through the C ABI, against the oracle.

* The stages of Q = P A_H⁻¹ Pᵀ (hdd_coarse_grid_op): restriction and interpolation in FP64 to
  rounding level; the sine-transform coarse solve backward stable against A_H = K_H - k²H² I
  (residual a small multiple of eps of the work precision) and against the oracle's banded LU
  of the same A_H within eps times cond(A_H) (both sides carry that error); coarse grids of 31,
  64 and 99 unknowns a side (one ragged 32-wide transform tile, two full tiles, four with a
  ragged tail), c = 2 and 3, both diagonal directions.
* The hybrid preconditioner z = Q v + M_RAS⁻¹(v - A Q v) with direct local solves: a fixed
  linear map, FP64 on both sides.
* Whole two-level solves: the plain FP64 form against the oracle's two-level solve (outer
  iterations ±1, solution within 1e-5), the default complex64 form (+10 %), a batch of two
  right-hand sides against single solves, and the k=200 bench workload at all 408,321 nodes
  against the oracle's stored two-level solve.
* Refusals: a factor that does not divide N, the impedance problem, two_level before set-up.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def _dev(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _maxrel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-300)


def _close(a, b, tol):
    return _rel(a, b) < tol and _maxrel(a, b) < tol


def _spectrum_AH(N, c, k):
    """(max |D|, cond(A_H)) from the closed-form spectrum of the lumped coarse operator."""
    Nc = N // c
    lam = 4 * np.sin(np.arange(1, Nc) * np.pi / (2 * Nc)) ** 2
    d = np.abs(lam[:, None] + lam[None, :] - (k / Nc) ** 2)
    return float(d.max()), float(d.max() / d.min())


# (N, k, c, diag): coarse m = N/c - 1 = 99, 31, 64
STAGE_CASES = [(200, 60.0, 2, 0), (96, 30.0, 3, 1), (130, 40.0, 2, 1)]


@pytest.mark.parametrize("N,k,c,diag", STAGE_CASES)
@pytest.mark.parametrize("prec", [128, 64])
def test_coarse_grid_stages_match_oracle(oracle_mod, N, k, c, diag, prec):
    _torch()
    from paper_2103_17081_gb300 import Solver
    s = Solver(0).assemble(k, N, diag=diag)
    s.setup_dd(2, 2, 2)
    s.setup_coarse_grid(c)
    p = oracle_mod.Problem(N, k, diag=diag)
    p.setup_dd(1, 1, 1, [0, N], [0, N])
    p.setup_coarse_grid(c)
    mm = (N // c - 1) ** 2
    assert s.coarse_grid_size == mm == p.cg_n()
    v = W.random_complex(p.n, 11)
    y = W.random_complex(mm, 12)
    eps = 2.0 ** -52 if prec == 128 else 2.0 ** -23
    # restriction and interpolation: FP64 arithmetic, the coarse side rounded to the work precision
    grid_tol = 1e-14 if prec == 128 else 2 * eps
    assert _close(s.coarse_grid_op("R", _dev(v), prec).cpu().numpy(), p.cg_Pt(v), grid_tol)
    assert _close(s.coarse_grid_op("P", _dev(y), prec).cpu().numpy(), p.cg_P(y), grid_tol)
    # A_H⁻¹ by orthogonal transforms is backward stable: the residual against A_H = K_H - k²H² I
    # (K_H assembled on the coarse mesh by the oracle) is a small multiple of eps, whatever the
    # conditioning; the forward error against the oracle's banded LU is within eps·cond(A_H)
    m = N // c - 1
    dmax, cond = _spectrum_AH(N, c, k)
    AH = oracle_mod.Problem(N // c, k, diag=diag).matrix("K") - (k * c / N) ** 2 * np.eye(mm)
    xs = s.coarse_grid_op("S", _dev(y), prec).cpu().numpy()
    back = np.linalg.norm(AH @ xs - y) / (dmax * np.linalg.norm(xs) + np.linalg.norm(y))
    assert back < 20 * np.sqrt(m) * eps, back
    ctol = max(50 * eps * cond * np.sqrt(m), 1e-13)
    xo = p.cg_solve(y)
    assert _close(xs, xo, ctol)
    # all three stages: Q v
    qo = p.cg_P(p.cg_solve(p.cg_Pt(v)))
    assert _close(s.coarse_grid_op("RSP", _dev(v), prec).cpu().numpy(), qo, ctol)


def test_hybrid_preconditioner_matches_oracle(oracle_mod):
    _torch()
    from paper_2103_17081_gb300 import Solver
    w = W.custom(20.0, 64, 4, 2)
    s = Solver.from_workload(w, exact=True).setup_coarse_grid(2)
    p = oracle_mod.from_workload(w, exact=True)
    p.setup_coarse_grid(2)
    v = W.random_complex(p.n, 5)
    A = p.matrix("A")
    qv = p.cg_P(p.cg_solve(p.cg_Pt(v)))
    zo = qv + p.ras_apply(v - A @ qv, 0.0)[0]
    zg, _ = s.ras_apply(_dev(v), inner_tol=0.0, inner_prec=128, two_level=1)
    assert _close(zg.cpu().numpy(), zo, 1e-11)
    # and the one-level application differs from it
    z1, _ = s.ras_apply(_dev(v), inner_tol=0.0, inner_prec=128)
    assert _rel(z1.cpu().numpy(), zo) > 1e-3


@pytest.mark.parametrize("prec", [128, 64])
def test_two_level_solve_matches_oracle(oracle_mod, prec):
    """k = 20, N = 64 (kh = 0.3125), 4x4 subdomains, inner tolerance 1e-2."""
    _torch()
    from paper_2103_17081_gb300 import Solver
    w = W.custom(20.0, 64, 4, 2)
    s = Solver.from_workload(w).setup_coarse_grid(2)
    p = oracle_mod.from_workload(w)
    p.setup_coarse_grid(2)
    fo = p.rhs(w.rhs[0])
    xo, so = p.solve(fo, two_level=1)
    f = s.build_rhs(w.rhs[0])
    x, st = s.solve(f, inner_prec=prec, outer_reorth32=int(prec == 64), two_level=1)
    xg = x.cpu().numpy()
    A = p.matrix("A")
    assert np.linalg.norm(fo - A @ xg) <= 1.0001e-6 * np.linalg.norm(fo)
    assert _close(xg, xo, 1e-5)
    if prec == 128:
        assert abs(st["outer_its"] - so["outer_its"]) <= 1
        hg, ho = np.array(st["res_history"]), np.array(so["res_history"])
        assert np.allclose(hg[:5], ho[:5], rtol=1e-6, atol=0)
    else:
        assert st["outer_its"] <= 1.1 * so["outer_its"] + 1
    # the coarse space pays: the one-level solve of the same problem takes more iterations
    _, s1 = s.solve(f, inner_prec=prec, outer_reorth32=int(prec == 64))
    assert st["outer_its"] < s1["outer_its"]


def test_two_level_batch_matches_single_solves():
    """Two right-hand sides in one batch (lockstep outer iterations; the one that converges first
    is masked out of the coarse-grid kernels) against each solved alone, plain FP64 form."""
    _torch()
    from paper_2103_17081_gb300 import Solver
    w = W.custom(20.0, 64, 4, 2)
    specs = [W.RHSSpec([W.PointSource(0.5, 0.5)]), W.RHSSpec([W.PointSource(0.3, 0.7, 2.0)])]
    kw = dict(inner_prec=128, outer_reorth32=0, two_level=1)
    s1 = Solver.from_workload(w).setup_coarse_grid(2)
    singles = []
    for sp in specs:
        x, st = s1.solve(s1.build_rhs(sp), **kw)
        singles.append((x.cpu().numpy(), st["outer_its"]))
    s2 = Solver.from_workload(w)
    s2.setup_batch(2)
    s2.setup_coarse_grid(2)
    fb = s2.build_rhs_batch(specs)
    xb, stb = s2.solve(fb, **kw)
    xb = xb.cpu().numpy().reshape(2, -1)
    assert stb["outer_its"] == max(it for _, it in singles)
    for r in range(2):
        assert _close(xb[r], singles[r][0], 1e-12)


def test_k200_two_level_full_size_against_stored_oracle():
    """The bench workload (k=200, N=640, 8x8 subdomains) with the two-level preconditioner in the
    default form, at all 408,321 nodes against the oracle's two-level solve stored by
    tests/golden/make_k200_reference.py k200tl: outer iterations within +10 %, every node within
    1e-5 of max|x|, and the 2-norm within 1e-5 relative."""
    torch = _torch()
    from paper_2103_17081_gb300 import Solver
    ref = json.load(open(os.path.join(GOLD, "k200tl_oracle.json")))
    xr = np.load(os.path.join(GOLD, "k200tl_oracle_x.npy"))
    assert ref["two_level"] == 1 and ref["coarse_factor"] == 2
    w = W.make("k200")
    s = Solver.from_workload(w).setup_coarse_grid(2)
    f = s.build_rhs(w.rhs[0])
    x, st = s.solve(f, outer_tol=w.outer_tol, inner_tol=w.inner_tol, two_level=1)
    r = f - s.apply_A(x)
    assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(f)) <= 1.0001e-6
    assert st["outer_its"] <= 1.1 * ref["outer_its"]
    xg = x.cpu().numpy()
    assert float(np.max(np.abs(xg.imag))) == 0.0
    assert _close(xg.real, xr, 1e-5), (_rel(xg.real, xr), _maxrel(xg.real, xr))


def test_coarse_grid_refusals():
    _torch()
    from paper_2103_17081_gb300 import HDDError, Solver
    s = Solver(0).assemble(20.0, 64)
    s.setup_dd(2, 2, 2).setup_deflation()
    f = s.build_rhs(W.RHSSpec([W.PointSource(0.5, 0.5)]))
    with pytest.raises(HDDError) as e:
        s.solve(f, two_level=1)                 # not set up
    assert e.value.code == 2
    with pytest.raises(HDDError) as e:
        s.setup_coarse_grid(3)                  # 3 does not divide 64
    assert e.value.code == 1
    with pytest.raises(HDDError) as e:
        s.coarse_grid_op("RSP", f)              # not set up
    assert e.value.code == 2
    s.setup_coarse_grid(2)
    x, st = s.solve(f, two_level=1)
    assert st["status_code"] == 0
    q = Solver(0).assemble(20.0, 64, bc=1)
    with pytest.raises(HDDError) as e:
        q.setup_coarse_grid(2)                  # impedance problem
    assert e.value.code == 1
