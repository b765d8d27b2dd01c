"""Pins of the oracle's two-level variant (grid coarse space), CPU only.

The variant follows the paper's stated next step (§4: a coarse space for the RAS
preconditioner) with the published grid coarse space: P1 on a coarser mesh of the same
triangulation (H = c h), P1 interpolation P, restriction Pᵀ, the coarse operator rediscretised
on that mesh with its mass matrix lumped, and the hybrid combination z = Q v + M_RAS⁻¹(v − A Q v),
Q = P A_H⁻¹ Pᵀ.  Pinned against facts that do not restate the code:

* nested P1 spaces: Pᵀ K_h P = K_H and Pᵀ M_h P = M_H, with K_H and M_H assembled element by
  element on the coarse mesh by an independent oracle problem (a wrong interpolation weight,
  diagonal direction or index fails them);
* the lumped coarse operator is K_H − k² H² I (the P1 mass rows sum to H² at interior nodes), so
  its inverse maps the discrete sine mode (p, q) to itself divided by
  4 sin²(pπH/2) + 4 sin²(qπH/2) − k²H²;
* with one subdomain and exact local solves the preconditioner is A⁻¹ whatever Q is, so FGMRES
  stops after one iteration;
* the coarse correction lowers the outer iteration count (the purpose of a coarse space).
"""
import numpy as np
import pytest

import workloads as W


def _dense_P(p):
    nH = p.cg_n()
    cols = []
    for t in range(nH):
        e = np.zeros(nH, dtype=np.complex128)
        e[t] = 1.0
        cols.append(p.cg_P(e).real)
    return np.array(cols).T


@pytest.mark.parametrize("N,c,diag", [(8, 2, 0), (8, 2, 1), (12, 3, 0), (12, 2, 1)])
def test_galerkin_identities_of_nested_p1(oracle_mod, N, c, diag):
    k = 7.0
    p = oracle_mod.Problem(N, k, diag=diag)
    p.setup_dd(1, 1, 1, [0, N], [0, N])
    p.setup_coarse_grid(c)
    q = oracle_mod.Problem(N // c, k, diag=diag)
    P = _dense_P(p)
    assert P.shape == ((N - 1) ** 2, (N // c - 1) ** 2)
    Kh, Mh = p.matrix("K").toarray(), p.matrix("M").toarray()
    KH, MH = q.matrix("K").toarray(), q.matrix("M").toarray()
    np.testing.assert_allclose(P.T @ Kh @ P, KH, atol=1e-13)
    np.testing.assert_allclose(P.T @ Mh @ P, MH, atol=1e-16)
    # restriction is the transpose of interpolation
    v = W.random_complex(p.n, 3)
    np.testing.assert_allclose(p.cg_Pt(v), P.T @ v, atol=1e-14)


@pytest.mark.parametrize("diag", [0, 1])
def test_lumped_coarse_operator_spectrum(oracle_mod, diag):
    N, c, k = 16, 2, 11.0
    p = oracle_mod.Problem(N, k, diag=diag)
    p.setup_dd(1, 1, 1, [0, N], [0, N])
    p.setup_coarse_grid(c)
    Nc = N // c
    H = 1.0 / Nc
    m = Nc - 1
    x = np.arange(1, Nc)
    for (pp, qq) in [(1, 1), (2, 5), (7, 3), (4, 4)]:
        s = np.outer(np.sin(qq * np.pi * x * H), np.sin(pp * np.pi * x * H)).ravel()   # x fastest
        lam = 4 * np.sin(pp * np.pi * H / 2) ** 2 + 4 * np.sin(qq * np.pi * H / 2) ** 2 - (k * H) ** 2
        u = p.cg_solve(s.astype(np.complex128))
        np.testing.assert_allclose(u.real, s / lam, rtol=1e-11, atol=1e-13)
        assert np.max(np.abs(u.imag)) == 0.0
    assert p.cg_n() == m * m


def test_one_subdomain_exact_local_solve_converges_in_one_iteration(oracle_mod):
    w = W.custom(9.0, 16, 1, 1)
    p = oracle_mod.from_workload(w, exact=True)
    p.setup_coarse_grid(2)
    f = p.rhs(w.rhs[0])
    x, st = p.solve(f, inner_tol=0.0, two_level=1, outer_tol=1e-10)
    assert st["outer_its"] == 1
    A = p.matrix("A")
    assert np.linalg.norm(f - A @ x) <= 1e-10 * np.linalg.norm(f)


def test_coarse_correction_lowers_outer_iterations(oracle_mod):
    """k = 20, N = 64: kh = 0.3125 as in the paper's runs (20 points per wavelength, so 10 on the
    coarse grid H = 2h), 4x4 subdomains, default inner tolerance (one level: 39 outer iterations,
    two levels: 11)."""
    w = W.custom(20.0, 64, 4, 2)
    p = oracle_mod.from_workload(w)
    p.setup_coarse_grid(2)
    f = p.rhs(w.rhs[0])
    x1, s1 = p.solve(f)
    x2, s2 = p.solve(f, two_level=1)
    A = p.matrix("A")
    assert np.linalg.norm(f - A @ x2) <= 1.0001e-6 * np.linalg.norm(f)
    assert s2["outer_its"] < s1["outer_its"], (s2["outer_its"], s1["outer_its"])
    assert np.linalg.norm(x2 - x1) <= 1e-5 * np.linalg.norm(x1)


def test_coarse_grid_refuses_bad_settings(oracle_mod):
    p = oracle_mod.Problem(15, 5.0)
    with pytest.raises(oracle_mod.OracleError):
        p.setup_coarse_grid(2)            # 2 does not divide 15
    q = oracle_mod.Problem(16, 5.0, bc=1)
    with pytest.raises(oracle_mod.OracleError):
        q.setup_coarse_grid(2)            # the impedance variant has no coarse grid here
    w = W.make("tiny")
    r = oracle_mod.from_workload(w)
    with pytest.raises(oracle_mod.OracleError):
        r.solve(r.rhs(w.rhs[0]), two_level=1)     # not set up


def test_first_iterate_is_the_hybrid_preconditioner_direction(oracle_mod):
    """With exact local solves the preconditioner is the fixed linear map
    B v = Q v + M_RAS⁻¹(v − A Q v), and one FGMRES step from x0 = 0 returns x1 = α B f with the
    least-squares α = (A B f)ᴴ f / ‖A B f‖².  B f is composed here from the separately pinned
    pieces (P, Pᵀ, A_H⁻¹, the one-level RAS apply and A), so a wrong sign, a dropped term or
    a swapped order in the hybrid step fails."""
    w = W.custom(20.0, 64, 4, 2)
    p = oracle_mod.from_workload(w, exact=True)
    p.setup_coarse_grid(2)
    A = p.matrix("A")
    f = p.rhs(w.rhs[0])
    Qf = p.cg_P(p.cg_solve(p.cg_Pt(f)))
    Bf = Qf + p.ras_apply(f - A @ Qf, 0.0)[0]
    ABf = A @ Bf
    alpha = np.vdot(ABf, f) / np.vdot(ABf, ABf)
    x1, st = p.solve(f, outer_maxit=1, inner_tol=0.0, two_level=1, raise_on_error=False)
    assert st["outer_its"] == 1
    np.testing.assert_allclose(x1, alpha * Bf, rtol=0, atol=1e-11 * np.max(np.abs(Bf * alpha)))
    # and the one-level step is the plain RAS direction, which differs
    x1r, _ = p.solve(f, outer_maxit=1, inner_tol=0.0, raise_on_error=False)
    assert np.linalg.norm(x1r - x1) > 1e-3 * np.linalg.norm(x1)
