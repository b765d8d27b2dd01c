"""Pins of the oracle's Krylov solvers (§3): deflated GMRES per subdomain and outer FGMRES+RAS.

Brute force: on tiny problems the k-th GMRES iterate must minimise the residual over the Krylov
space (dense least squares over an explicitly built Krylov basis), and the k-th FGMRES iterate
with a fixed (exact) RAS preconditioner must minimise ||f - A M⁻¹ y|| the same way.  Plus: exact
limits (tight inner tolerance = direct solve), the one-subdomain special cases, agreement with a
dense direct solve of the global system, and the real-data invariant Im u = 0.
"""
import numpy as np
import pytest

import workloads as W


def _krylov_min_residual(Aop, b, k):
    """min over u in K_k(Aop, b) of ||b - Aop u||, from a dense orthonormal Krylov basis."""
    n = b.shape[0]
    K = np.zeros((n, k), dtype=complex)
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = Aop @ v
    Q, _ = np.linalg.qr(K)
    AQ = Aop @ Q
    y, *_ = np.linalg.lstsq(AQ, b, rcond=None)
    return np.linalg.norm(b - AQ @ y)


def _tiny(oracle_mod, N=14, k=9.0, S=2, overlap=1):
    w = W.custom(k, N, S, overlap)
    p = oracle_mod.Problem(w.N, w.k)
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    p.setup_deflation()
    p.setup_exact()
    return p, w


def test_inner_gmres_is_krylov_minimiser(oracle_mod):
    p, w = _tiny(oracle_mod)
    s = 0
    n = p.sub_n(s)
    assert n <= 64
    As = p.sub_A(s).toarray()
    # dense P A and P f from the oracle's own P applied to unit vectors
    P = np.column_stack([p.sub_apply_P(s, np.eye(n, dtype=complex)[:, c]) for c in range(n)])
    f = W.random_complex(n, 21)
    PA, Pf = P @ As, P @ f
    for k in (1, 2, 4, 7):
        x, its = p.sub_solve(s, f, tol=1e-30, restart=40, maxit=k)
        assert its == k
        # completion makes the true residual equal the deflated one
        got = np.linalg.norm(f - As @ x)
        ref = _krylov_min_residual(PA, Pf, k)
        assert got == pytest.approx(ref, rel=1e-8, abs=1e-13 * np.linalg.norm(f))


def test_inner_restart_and_tight_tolerance_reach_direct(oracle_mod):
    p, w = _tiny(oracle_mod, N=20, k=12.0)
    for s in range(p.nsub):
        f = W.random_complex(p.sub_n(s), 30 + s)
        xd = np.linalg.solve(p.sub_A(s).toarray(), f)
        x, its = p.sub_solve(s, f, tol=1e-13, restart=5, maxit=2000)
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
        assert np.linalg.norm(p.sub_solve_exact(s, f) - xd) <= 1e-11 * np.linalg.norm(xd)


def test_inner_tolerance_is_met_on_true_residual(oracle_mod):
    p, w = _tiny(oracle_mod, N=30, k=20.0)
    for tol in (1e-1, 1e-2, 1e-5):
        f = W.random_complex(p.sub_n(0), 7)
        x, its = p.sub_solve(0, f, tol=tol, restart=30, maxit=1000)
        Pf = p.sub_apply_P(0, f)
        res = np.linalg.norm(f - p.sub_A(0) @ x)
        assert res <= tol * np.linalg.norm(Pf) * (1 + 1e-8)


def test_warm_start_counts_relative_to_Pf(oracle_mod):
    """A perfect initial guess needs no iterations (tolerance relative to ||P f||)."""
    p, w = _tiny(oracle_mod, N=20, k=12.0)
    f = W.random_complex(p.sub_n(0), 3)
    xd = p.sub_solve_exact(0, f)
    x, its = p.sub_solve(0, f, tol=1e-6, x0=xd)
    assert its == 0 and np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_fgmres_is_krylov_minimiser_with_exact_ras(oracle_mod):
    p, w = _tiny(oracle_mod, N=12, k=8.0, S=2)
    n = p.n
    A = p.matrix("A").toarray()
    Mi = np.column_stack([p.ras_apply(np.eye(n, dtype=complex)[:, c], inner_tol=0.0)[0]
                          for c in range(n)])
    f = W.random_complex(n, 4)
    AM = A @ Mi
    for k in (1, 3, 6):
        x, st = p.solve(f, outer_tol=1e-30, outer_restart=50, outer_maxit=k, inner_tol=0.0,
                        raise_on_error=False)
        assert st["outer_its"] == k
        got = np.linalg.norm(f - A @ x)
        ref = _krylov_min_residual(AM, f, k)
        assert got == pytest.approx(ref, rel=1e-8)


def test_one_subdomain_special_cases(oracle_mod):
    w = W.custom(10.0, 20, 1, 1)
    p = oracle_mod.Problem(w.N, w.k)
    p.setup_dd(1, 1, 1, [0, 20], [0, 20])
    p.setup_deflation()
    p.setup_exact()
    f = p.rhs(w.rhs[0])
    x, st = p.solve(f, inner_tol=0.0)
    assert st["outer_its"] == 1
    # with inner tolerance τ the first outer residual is at most τ ||P f|| / ||f||
    tau = 1e-2
    x, st = p.solve(f, outer_tol=1e-30, outer_maxit=1, inner_tol=tau, raise_on_error=False)
    Pf = p.sub_apply_P(0, f)
    assert st["res_history"][0] <= tau * np.linalg.norm(Pf) / np.linalg.norm(f) * (1 + 1e-8)


def test_tiny_workload_matches_direct_solve(oracle_mod):
    import scipy.sparse.linalg as spla
    w = W.make("tiny")
    p = oracle_mod.from_workload(w)
    f = p.rhs(w.rhs[0])
    x, st = p.solve(f, outer_tol=1e-10, inner_tol=1e-2)
    xd = spla.spsolve(p.matrix("A").tocsc(), f)
    A = p.matrix("A")
    assert np.linalg.norm(f - A @ x) <= 1e-10 * np.linalg.norm(f) * (1 + 1e-6)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert np.all(x.imag == 0.0)             # real data stays real


def test_tight_inner_reproduces_direct_ras_history(oracle_mod):
    w = W.custom(16.0, 40, 2, 2)
    p = oracle_mod.Problem(w.N, w.k)
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    p.setup_deflation()
    p.setup_exact()
    f = p.rhs(w.rhs[0])
    _, st_lu = p.solve(f, inner_tol=0.0)
    _, st_it = p.solve(f, inner_tol=1e-13)
    n = min(20, len(st_lu["res_history"]))
    h1, h2 = st_lu["res_history"][:n], st_it["res_history"][:n]
    assert np.max(np.abs(h1 - h2) / h1) < 1e-8
    assert st_lu["outer_its"] == st_it["outer_its"]


def test_inner_counts_fall_as_tolerance_loosens(oracle_mod):
    """Trend of Tables 2–4: looser inner tolerance, fewer inner and not fewer outer iterations."""
    w = W.custom(20.0, 60, 2, 1)
    p = oracle_mod.from_workload(w)
    f = p.rhs(w.rhs[0])
    res = {}
    for tol in (1e-10, 1e-5, 1e-2):
        _, st = p.solve(f, inner_tol=tol)
        res[tol] = (st["outer_its"], st["inner_its_avg"])
    assert res[1e-10][1] > res[1e-5][1] > res[1e-2][1]
    assert res[1e-2][0] >= res[1e-10][0]


def test_nonfinite_rhs_is_reported(oracle_mod):
    w = W.make("tiny")
    p = oracle_mod.from_workload(w)
    f = p.rhs(w.rhs[0])
    f[5] = np.nan
    with pytest.raises(oracle_mod.OracleError):
        p.solve(f)


def test_outer_cgs2_projects_out_an_orthonormal_basis(oracle_mod):
    """For orthonormal V: the result is orthogonal to V, w_in = w' + V h exactly in exact
    arithmetic (here to rounding), h = Vᴴ w_in, and the returned value is ||w'||."""
    rng = np.random.default_rng(8)
    n, nv = 300, 12
    V, _ = np.linalg.qr(rng.standard_normal((n, nv)) + 1j * rng.standard_normal((n, nv)))
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    wp, h, r = oracle_mod.cgs2(V, w)
    assert np.linalg.norm(V.conj().T @ wp) <= 1e-14 * np.linalg.norm(w)
    assert np.linalg.norm(w - (wp + V @ h)) <= 1e-14 * np.linalg.norm(w)
    assert np.allclose(h, V.conj().T @ w, rtol=0, atol=1e-13 * np.linalg.norm(w))
    assert r == pytest.approx(np.linalg.norm(wp), rel=1e-14)
    # a vector already in span(V) leaves (almost) nothing
    wp, h, r = oracle_mod.cgs2(V, V @ h)
    assert r <= 1e-14 * np.linalg.norm(h)
