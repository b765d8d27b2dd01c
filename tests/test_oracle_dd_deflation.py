"""Pins of the oracle's decomposition (Eq. 3, §3) and two-level deflation (Eq. 4, Eq. 5).

Checked against: the hand-written 1D deflation matrix from the paper's Bézier stencil
(tests/golden/z1d_nx5_nx6.txt), the partition of unity, dense linear algebra (numpy) for
E = ZᵀAZ, the deflation invariant P A Z = 0, and the completion identity of the deflated solve.
"""
import os

import numpy as np
import pytest

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_z1d():
    mats, cur, nx = {}, None, None
    for line in open(os.path.join(GOLD, "z1d_nx5_nx6.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("nx"):
            if cur:
                mats[nx] = np.array(cur, dtype=float) / 8.0
            nx, cur = int(line.split()[1]), []
            continue
        cur.append([float(t) for t in line.split()])
    mats[nx] = np.array(cur, dtype=float) / 8.0
    return mats


def _problem(oracle_mod, N=24, k=15.0, S=2, Sy=None, overlap=2, ifx=None, ify=None):
    w = W.custom(k, N, S, overlap, Sy=Sy, ifx=ifx, ify=ify)
    p = oracle_mod.Problem(w.N, w.k)
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    return p, w


def test_partition_of_unity_and_boxes(oracle_mod):
    for (N, S, ov) in [(32, 2, 2), (30, 3, 1), (41, 4, 3)]:
        p, w = _problem(oracle_mod, N=N, S=S, overlap=ov)
        owned = np.zeros(p.n, dtype=int)
        for s in range(p.nsub):
            b = p.box(s)
            assert b["ix0"] <= b["ox0"] <= b["ox1"] <= b["ix1"]
            assert b["iy0"] <= b["oy0"] <= b["oy1"] <= b["iy1"]
            for j in range(b["oy0"], b["oy1"] + 1):
                for i in range(b["ox0"], b["ox1"] + 1):
                    owned[(i - 1) + (j - 1) * (N - 1)] += 1
        assert np.all(owned == 1)          # Σ R_jᵀ D_j R_j = I


def test_box_widths_k200_geometry(oracle_mod):
    w = W.make("k200")
    p = oracle_mod.Problem(w.N, 0.0)
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    widths = sorted({p.box(s)["nx"] for s in range(p.nsub)})
    assert widths == [81, 83]              # 80-cell subdomains, 2 layers of overlap


def test_local_matrix_is_submatrix(oracle_mod):
    p, w = _problem(oracle_mod, N=20, S=3)
    A = p.matrix("A").toarray()
    for s in range(p.nsub):
        b = p.box(s)
        idx = [(i - 1) + (j - 1) * (w.N - 1) for j in range(b["iy0"], b["iy1"] + 1)
               for i in range(b["ix0"], b["ix1"] + 1)]
        assert np.array_equal(p.sub_A(s).toarray(), A[np.ix_(idx, idx)])


def test_Z_matches_handwritten_stencil(oracle_mod):
    gold = _read_z1d()
    # a box of nx x ny = 5 x 6 nodes: Z must equal Zy ⊗ Zx of the hand-written 1D matrices
    p = oracle_mod.Problem(6, 1.0)
    p.setup_dd(1, 1, 1, [0, 6], [0, 6])     # one subdomain, box 5 x 5
    p.setup_deflation()
    Z = p.sub_Z(0).toarray()
    assert np.array_equal(Z, np.kron(gold[5], gold[5]))
    p2 = oracle_mod.Problem(7, 1.0)
    p2.setup_dd(1, 1, 1, [0, 7], [0, 7])    # box 6 x 6
    p2.setup_deflation()
    assert np.array_equal(p2.sub_Z(0).toarray(), np.kron(gold[6], gold[6]))


def test_Z_rank_E_symmetric_and_galerkin(oracle_mod):
    p, w = _problem(oracle_mod, N=30, k=18.0, S=2, Sy=3)
    p.setup_deflation()
    for s in range(p.nsub):
        Z = p.sub_Z(s).toarray()
        b = p.box(s)
        assert Z.shape == (b["nx"] * b["ny"], (b["nx"] // 2) * (b["ny"] // 2))
        assert np.linalg.matrix_rank(Z) == Z.shape[1]
        E = p.E_dense(s)
        As = p.sub_A(s).toarray()
        assert np.max(np.abs(E - Z.T @ As @ Z)) < 1e-13 * np.max(np.abs(E))
        assert np.max(np.abs(E - E.T)) <= 1e-15 * np.max(np.abs(E))
        kl, ku = p.E_band(s)
        assert kl == ku == 2 * (b["nx"] // 2) + 2   # 5x5 coarse stencil, x fastest


def test_coarse_solve_and_band_lu(oracle_mod):
    p, w = _problem(oracle_mod, N=30, k=18.0, S=2)
    p.setup_deflation()
    E = p.E_dense(0)
    y = W.random_complex(E.shape[0], 5)
    x = p.coarse_solve(0, y)
    assert np.max(np.abs(x - np.linalg.solve(E.astype(complex), y))) < 1e-11 * np.max(np.abs(x))
    # banded LU with pivoting on a random band matrix whose pivots must move
    rng = np.random.default_rng(3)
    m, kl, ku = 40, 3, 2
    D = np.zeros((m, m))
    for r in range(m):
        for c in range(max(0, r - kl), min(m, r + ku + 1)):
            D[r, c] = rng.uniform(-1, 1)
    D[np.arange(m), np.arange(m)] *= 1e-3          # force row interchanges
    Wd = 2 * kl + ku + 1
    ab = np.zeros((m, Wd))
    for r in range(m):
        for c in range(max(0, r - kl), min(m, r + ku + 1)):
            ab[r, c - r + kl] = D[r, c]
    ab, piv = oracle_mod.band_lu(ab, m, kl, ku)
    assert np.any(piv != np.arange(m))
    b = W.random_complex(m, 9)
    xb = oracle_mod.band_solve(ab, piv, m, kl, ku, b)
    assert np.max(np.abs(D @ xb - b)) < 1e-11 * np.max(np.abs(xb))


def test_deflation_invariant_PAZ_zero(oracle_mod):
    p, w = _problem(oracle_mod, N=40, k=25.0, S=2)
    p.setup_deflation()
    for s in range(p.nsub):
        Z = p.sub_Z(s).toarray()
        As = p.sub_A(s).toarray()
        worst = 0.0
        for c in range(0, Z.shape[1], 7):
            paz = p.sub_apply_PA(s, Z[:, c].astype(complex))
            worst = max(worst, np.linalg.norm(paz) / np.linalg.norm(As @ Z[:, c]))
        assert worst < 1e-12


def test_projection_properties(oracle_mod):
    """P² = P and Zᵀ P = 0 (P = I - A Q projects onto the complement of range(AZ))."""
    p, w = _problem(oracle_mod, N=30, k=18.0, S=2)
    p.setup_deflation()
    v = W.random_complex(p.sub_n(1), 11)
    Pv = p.sub_apply_P(1, v)
    assert np.linalg.norm(p.sub_apply_P(1, Pv) - Pv) < 1e-12 * np.linalg.norm(Pv)
    assert np.linalg.norm(p.sub_apply_Zt(1, Pv)) < 1e-12 * np.linalg.norm(p.sub_apply_Zt(1, v))


def test_completion_identity(oracle_mod):
    """x = u + Q(f - A u) gives A x - f = -P(f - A u): the deflated residual is the true one."""
    p, w = _problem(oracle_mod, N=30, k=18.0, S=2)
    p.setup_deflation()
    s = 0
    n = p.sub_n(s)
    f = W.random_complex(n, 1)
    u = W.random_complex(n, 2)
    As = p.sub_A(s)
    r = f - As @ u
    Zt_r = p.sub_apply_Zt(s, r)
    x = u + p.sub_apply_Z(s, p.coarse_solve(s, Zt_r))
    lhs = As @ x - f
    rhs = -p.sub_apply_P(s, r)
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(r)


def test_singular_pivot_reported(oracle_mod):
    """A column with no non-zero pivot candidate is reported as singular (no NaN is produced)."""
    m, kl, ku = 6, 1, 1
    ab = np.zeros((m, 2 * kl + ku + 1))
    for r in range(m):
        ab[r, kl] = 1.0
    ab[3, kl] = 0.0
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.band_lu(ab, m, kl, ku)
