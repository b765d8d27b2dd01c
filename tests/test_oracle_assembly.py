"""Pins of the oracle's P1 assembly (§2, Eq. 1–2) against closed forms.

The oracle assembles element by element; these tests check it against facts derived by hand
from the mathematics: the 7-point stencil of K - k²M on the SW–NE triangulation, the unit
partition of the mass matrix, the closed-form spectrum of the discrete Dirichlet Laplacian, and
second-order convergence to a manufactured solution.
"""
import math

import numpy as np
import pytest


def _entry(A, N, i, j, di, dj):
    r = (i - 1) + (j - 1) * (N - 1)
    c = (i + di - 1) + (j + dj - 1) * (N - 1)
    return A[r, c]


@pytest.mark.parametrize("diag", [0, 1])
def test_stencil_closed_form(oracle_mod, diag):
    N, k = 12, 7.0
    h = 1.0 / N
    p = oracle_mod.Problem(N, k, diag)
    A = p.matrix("A").toarray()
    kk = k * k * h * h
    # hand derivation: K = 5-point [4; -1 x4]; M = h²/12 [6; 1 at E,W,N,S and at the two
    # corners joined by the cell diagonals]; A = K - k² M.
    diag_nb = [(1, 1), (-1, -1)] if diag == 0 else [(1, -1), (-1, 1)]
    off_nb = [(1, -1), (-1, 1)] if diag == 0 else [(1, 1), (-1, -1)]
    for (i, j) in [(5, 5), (2, 3), (6, 9)]:
        assert _entry(A, N, i, j, 0, 0) == pytest.approx(4 - kk / 2, rel=1e-14)
        for d in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
            assert _entry(A, N, i, j, *d) == pytest.approx(-1 - kk / 12, rel=1e-14)
        for d in diag_nb:
            assert _entry(A, N, i, j, *d) == pytest.approx(-kk / 12, rel=1e-14)
        for d in off_nb:
            assert _entry(A, N, i, j, *d) == 0.0
    assert np.count_nonzero(np.abs(A[(4 - 1) + (4 - 1) * (N - 1)]) > 0) == 7


def test_symmetry_and_mass_partition(oracle_mod):
    N = 10
    p = oracle_mod.Problem(N, 3.0)
    A, M = p.matrix("A"), p.matrix("M")
    assert abs(A - A.T).max() == 0.0
    Md = M.toarray()
    h = 1.0 / N
    # each hat function integrates to h² (6 triangles of area h²/2, 1/3 each); away from the
    # boundary the whole row of M is present, so its sum is exactly that integral
    for (i, j) in [(3, 3), (5, 7)]:
        r = (i - 1) + (j - 1) * (N - 1)
        assert Md[r].sum() == pytest.approx(h * h, rel=1e-13)


def test_stiffness_spectrum_closed_form(oracle_mod):
    """K (k=0 stiffness) has eigenvalues 4 sin²(pπh/2) + 4 sin²(qπh/2), p,q = 1..N-1."""
    N = 12
    h = 1.0 / N
    p = oracle_mod.Problem(N, 0.0)
    ev = np.sort(np.linalg.eigvalsh(p.matrix("K").toarray()))
    ref = np.sort([4 * math.sin(a * math.pi * h / 2) ** 2 + 4 * math.sin(b * math.pi * h / 2) ** 2
                   for a in range(1, N) for b in range(1, N)])
    assert np.max(np.abs(ev - ref)) < 1e-12


def test_sine_eigenvectors(oracle_mod):
    """sin(pπx) sin(qπy) sampled on the nodes is an eigenvector of K."""
    N, pp, qq = 10, 2, 3
    h = 1.0 / N
    p = oracle_mod.Problem(N, 0.0)
    v = np.array([math.sin(pp * math.pi * i * h) * math.sin(qq * math.pi * j * h)
                  for j in range(1, N) for i in range(1, N)], dtype=complex)
    lam = 4 * math.sin(pp * math.pi * h / 2) ** 2 + 4 * math.sin(qq * math.pi * h / 2) ** 2
    assert np.max(np.abs(p.apply(v, "K") - lam * v)) < 1e-13


def test_manufactured_second_order(oracle_mod):
    """-Δu - k²u = f with u = sin πx sin πy: nodal error O(h²), observed rate in [1.9, 2.1]."""
    import scipy.sparse.linalg as spla
    k = 5.0
    errs, hs = [], []
    for N in (16, 32, 64, 128):
        p = oracle_mod.Problem(N, k)
        f = p.rhs_manufactured()
        u = spla.spsolve(p.matrix("A").tocsc(), f)
        h = 1.0 / N
        ex = np.array([math.sin(math.pi * i * h) * math.sin(math.pi * j * h)
                       for j in range(1, N) for i in range(1, N)])
        errs.append(np.max(np.abs(u - ex)))
        hs.append(h)
    rates = [math.log(errs[t] / errs[t + 1]) / math.log(hs[t] / hs[t + 1]) for t in range(3)]
    assert all(1.9 <= r <= 2.1 for r in rates), rates


def test_point_source_and_bump_load(oracle_mod):
    N = 20
    p = oracle_mod.Problem(N, 4.0)
    import workloads as W
    f = p.rhs(W.RHSSpec([W.PointSource(0.5, 0.5)]))
    c = (10 - 1) + (10 - 1) * (N - 1)
    assert f[c] == 1.0 and np.count_nonzero(f) == 1
    # clamping: a source on the boundary goes to the nearest interior node
    f2 = p.rhs(W.RHSSpec([W.PointSource(0.0, 1.0)]))
    assert f2[(1 - 1) + (N - 1 - 1) * (N - 1)] == 1.0
    # bump load is M g with g the nodal Gaussian (interior nodes)
    b = W.Bump(0.4, 0.6, 0.1)
    fb = p.rhs(W.RHSSpec([], [b]))
    h = 1.0 / N
    g = np.array([math.exp(-((i * h - 0.4) ** 2 + (j * h - 0.6) ** 2) / (2 * 0.01))
                  for j in range(1, N) for i in range(1, N)])
    assert np.max(np.abs(fb - p.matrix("M") @ g)) < 1e-15
