"""Pins of the oracle's impedance (Sommerfeld) variant: du/dn - i k u = 0 on all of the boundary.

The paper computes with the Dirichlet problem of Eq. 1 and notes in §3 that the solver (RAS with
GMRES, neither needing symmetry) is also meant for the non-symmetric Sommerfeld problem.  The
reading taken: the first-order absorbing condition on all four sides, every mesh node an unknown,
A = K - k²M - i k B with B the boundary mass matrix (complex symmetric, not Hermitian), local
matrices A_j = R_j A R_jᵀ (impedance rows kept where a box meets the physical boundary, Dirichlet
on its artificial sides), and the deflation matrix of Eq. 5 on each local node box.

Pinned against values fixed by the mathematics, not by the oracle's own formulas:
  - exact integrals of P1 functions: the boundary length and the moments of x and y over the
    boundary and over the square (the consistent P1 masses integrate these exactly);
  - the plane wave exp(i k (x cos θ + y sin θ)), an exact solution of the continuous problem
    with boundary data the test computes itself: the nodal error must fall like h² (a wrong sign
    of the i k B term, a missing side or a wrong boundary weight leaves an O(1) error);
  - the sine manufactured solution with its boundary datum;
  - the energy identity Im(uᴴ f) = -k uᴴ B u of the discrete solution (outgoing flux);
  - the mesh symmetries of a centred point source;
  - dense linear algebra (numpy) for the complex banded LU, E = ZᵀAZ and the coarse solve;
  - the partition of unity over all (N+1)² nodes; brute-force Krylov minimisation.
"""
import numpy as np
import pytest

import workloads as W


def _coords(p):
    """Nodal x and y of every unknown of an impedance problem."""
    N = p.N
    i = np.tile(np.arange(N + 1), N + 1)
    j = np.repeat(np.arange(N + 1), N + 1)
    return i / N, j / N


def _problem(oracle_mod, N=24, k=15.0, S=2, overlap=2, diag=0, defl=True, exact=False):
    w = W.custom(k, N, S, overlap, bc=1)
    p = oracle_mod.Problem(w.N, w.k, diag=diag, bc=1)
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    if defl:
        p.setup_deflation()
    if exact:
        p.setup_exact()
    return p, w


# -- assembly --------------------------------------------------------------------------------
@pytest.mark.parametrize("diag", [0, 1])
def test_boundary_mass_exact_moments(oracle_mod, diag):
    p = oracle_mod.Problem(12, 7.0, diag=diag, bc=1)
    assert p.n == 13 * 13
    B = p.matrix("B").toarray()
    X, Y = _coords(p)
    one = np.ones(p.n)
    assert np.array_equal(B, B.T)
    on_bnd = (X == 0) | (X == 1) | (Y == 0) | (Y == 1)
    assert np.all(B[~on_bnd] == 0) and np.all(B[:, ~on_bnd] == 0)
    # ∫_∂Ω 1 = 4, ∫ x = 1/2 + 1/2 + 0 + 1, ∫ x² = 1/3 + 1/3 + 0 + 1, ∫ x y = 0 + 1/2 + 0 + 1/2
    assert one @ B @ one == pytest.approx(4.0, rel=1e-13)
    assert one @ B @ X == pytest.approx(2.0, rel=1e-13)
    assert X @ B @ X == pytest.approx(5.0 / 3.0, rel=1e-13)
    assert X @ B @ Y == pytest.approx(1.0, rel=1e-13)
    assert Y @ B @ Y == pytest.approx(5.0 / 3.0, rel=1e-13)


@pytest.mark.parametrize("diag", [0, 1])
def test_all_node_stiffness_and_mass_moments(oracle_mod, diag):
    p = oracle_mod.Problem(10, 3.0, diag=diag, bc=1)
    K, M = p.matrix("K").toarray(), p.matrix("M").toarray()
    X, Y = _coords(p)
    one = np.ones(p.n)
    assert np.max(np.abs(K @ one)) < 1e-12              # constants are in the kernel of K
    assert X @ K @ X == pytest.approx(1.0, rel=1e-12)   # ∫ |∇x|²
    assert abs(X @ K @ Y) < 1e-12                       # ∫ ∇x·∇y
    assert Y @ K @ Y == pytest.approx(1.0, rel=1e-12)
    assert one @ M @ one == pytest.approx(1.0, rel=1e-13)
    assert one @ M @ X == pytest.approx(0.5, rel=1e-13)
    assert X @ M @ X == pytest.approx(1.0 / 3.0, rel=1e-13)
    assert X @ M @ Y == pytest.approx(0.25, rel=1e-13)


def test_A_is_complex_symmetric_with_boundary_damping(oracle_mod):
    k = 9.0
    p = oracle_mod.Problem(8, k, bc=1)
    A = p.matrix("A").toarray()
    K, M, B = (p.matrix(w).toarray() for w in ("K", "M", "B"))
    assert np.array_equal(A, A.T)
    assert not np.allclose(A, A.conj().T)
    assert np.allclose(A.real, K - k * k * M, rtol=0, atol=1e-14)
    assert np.allclose(A.imag, -k * B, rtol=0, atol=1e-14)


def _plane_wave_load(N, k, theta):
    """Load of the plane wave: f = 0 inside, the boundary datum g = du/dn - i k u of each side
    (linear interpolant along every boundary edge, ∫_e g_I φ_a = h/6 (2 g_a + g_b))."""
    h = 1.0 / N
    c, s = np.cos(theta), np.sin(theta)
    u = lambda x, y: np.exp(1j * k * (x * c + y * s))
    # outward normals: bottom (0,-1), top (0,1), left (-1,0), right (1,0)
    sides = [(lambda t: (t, 0.0), -1j * k * (s + 1.0)), (lambda t: (t, 1.0), 1j * k * (s - 1.0)),
             (lambda t: (0.0, t), -1j * k * (c + 1.0)), (lambda t: (1.0, t), 1j * k * (c - 1.0))]
    F = np.zeros((N + 1) * (N + 1), dtype=complex)
    idx = lambda x, y: int(round(x * N)) + int(round(y * N)) * (N + 1)
    for pos, fac in sides:
        for e in range(N):
            xa, ya = pos(e * h)
            xb, yb = pos((e + 1) * h)
            ga, gb = fac * u(xa, ya), fac * u(xb, yb)
            F[idx(xa, ya)] += h / 6.0 * (2 * ga + gb)
            F[idx(xb, yb)] += h / 6.0 * (2 * gb + ga)
    return F, u


def test_plane_wave_second_order(oracle_mod):
    import scipy.sparse.linalg as spla
    k, theta = 6.0, 0.3
    errs = []
    for N in (16, 32, 64, 128):
        p = oracle_mod.Problem(N, k, bc=1)
        F, u = _plane_wave_load(N, k, theta)
        uh = spla.spsolve(p.matrix("A").tocsc(), F)
        X, Y = _coords(p)
        ue = u(X, Y)
        errs.append(np.max(np.abs(uh - ue)) / np.max(np.abs(ue)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3
    assert np.all((rates > 1.8) & (rates < 2.3)), (errs, rates)


def test_manufactured_sine_second_order_with_impedance(oracle_mod):
    """The discrete L2 (RMS) nodal error falls like h²; the largest error sits at the corners,
    where the outward normal jumps, and its rate approaches 2 from below (1.5 to 1.75 for
    N = 16..256), so the max norm is only required to fall faster than h^1.4."""
    import scipy.sparse.linalg as spla
    rms, mx = [], []
    for N in (16, 32, 64):
        p = oracle_mod.Problem(N, 5.0, bc=1)
        uh = spla.spsolve(p.matrix("A").tocsc(), p.rhs_manufactured())
        X, Y = _coords(p)
        e = np.abs(uh - np.sin(np.pi * X) * np.sin(np.pi * Y))
        rms.append(np.sqrt(np.mean(e * e)))
        mx.append(e.max())
    r_rms = np.log2(np.array(rms[:-1]) / np.array(rms[1:]))
    r_max = np.log2(np.array(mx[:-1]) / np.array(mx[1:]))
    assert np.all((r_rms > 1.9) & (r_rms < 2.1)), (rms, r_rms)
    assert np.all(r_max > 1.4), (mx, r_max)


def test_point_source_snaps_to_any_node(oracle_mod):
    p = oracle_mod.Problem(10, 4.0, bc=1)
    f = p.rhs(W.RHSSpec([W.PointSource(0.0, 1.0, 2.0), W.PointSource(0.52, 0.48)]))
    assert f[p.node_index(0, 10)] == 2.0 and f[p.node_index(5, 5)] == 1.0
    assert np.count_nonzero(f) == 2


# -- decomposition and deflation -------------------------------------------------------------
def test_partition_of_unity_all_nodes(oracle_mod):
    for (N, S, ov) in [(32, 2, 2), (30, 3, 1), (41, 4, 3)]:
        w = W.custom(5.0, N, S, ov, bc=1)
        p = oracle_mod.Problem(N, 5.0, bc=1)
        p.setup_dd(S, S, ov, w.ifx, w.ify)
        owned = np.zeros(p.n, dtype=int)
        for s in range(p.nsub):
            b = p.box(s)
            px, py = s % S, s // S
            assert b["ix0"] == (0 if px == 0 else w.ifx[px] - ov + 1)
            assert b["ix1"] == (N if px == S - 1 else w.ifx[px + 1] + ov - 1)
            for j in range(b["oy0"], b["oy1"] + 1):
                for i in range(b["ox0"], b["ox1"] + 1):
                    owned[p.node_index(i, j)] += 1
        assert np.all(owned == 1)          # Σ R_jᵀ D_j R_j = I over all (N+1)² nodes


def test_local_matrix_is_complex_submatrix(oracle_mod):
    p, w = _problem(oracle_mod, N=16, k=10.0, S=2, overlap=2, defl=False)
    A = p.matrix("A").toarray()
    for s in range(p.nsub):
        b = p.box(s)
        g = [p.node_index(i, j) for j in range(b["iy0"], b["iy1"] + 1)
             for i in range(b["ix0"], b["ix1"] + 1)]
        As = p.sub_A(s).toarray()
        assert np.array_equal(As, A[np.ix_(g, g)])
        assert np.any(As.imag != 0)        # every box of a 2x2 split meets the boundary


def test_complex_band_lu_against_dense(oracle_mod):
    rng = np.random.default_rng(5)
    for (m, kl, ku) in [(40, 3, 2), (57, 5, 5), (9, 1, 4)]:
        D = np.zeros((m, m), dtype=complex)
        for r in range(m):
            for c in range(max(0, r - kl), min(m, r + ku + 1)):
                D[r, c] = rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1)
            D[r, r] *= 1e-3                # small diagonal: rows must be interchanged
        W_ = 2 * kl + ku + 1
        ab = np.zeros((m, W_), dtype=complex)
        for r in range(m):
            for c in range(max(0, r - kl), min(m, r + ku + 1)):
                ab[r, c - r + kl] = D[r, c]
        f, piv = oracle_mod.band_lu_z(ab, m, kl, ku)
        assert np.any(piv != np.arange(m))
        b = rng.uniform(-1, 1, m) + 1j * rng.uniform(-1, 1, m)
        x = oracle_mod.band_solve_z(f, piv, m, kl, ku, b)
        xd = np.linalg.solve(D, b)
        assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_E_is_galerkin_complex_symmetric_and_coarse_solve(oracle_mod):
    p, w = _problem(oracle_mod, N=24, k=15.0, S=2, overlap=2)
    for s in range(p.nsub):
        Z = p.sub_Z(s).toarray()
        As = p.sub_A(s).toarray()
        E = p.E_dense(s)
        Eref = Z.T @ As @ Z
        assert np.linalg.norm(E - Eref) <= 1e-13 * np.linalg.norm(Eref)
        assert np.array_equal(E, E.T) or np.linalg.norm(E - E.T) <= 1e-15 * np.linalg.norm(E)
        assert np.any(E.imag != 0)
        y = W.random_complex(p.sub_m(s), 40 + s)
        x = p.coarse_solve(s, y)
        xd = np.linalg.solve(Eref, y)
        assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_deflation_invariant_and_completion(oracle_mod):
    p, w = _problem(oracle_mod, N=24, k=15.0, S=2, overlap=2)
    s = 0
    Z = p.sub_Z(s).toarray()
    As = p.sub_A(s)
    AZ = As @ Z
    PAZ = np.column_stack([p.sub_apply_PA(s, Z[:, c].astype(complex)) for c in range(Z.shape[1])])
    assert np.linalg.norm(PAZ) <= 1e-12 * np.linalg.norm(AZ)
    f = W.random_complex(p.sub_n(s), 9)
    for tol in (1e-1, 1e-3, 1e-6):
        x, its = p.sub_solve(s, f, tol=tol)
        res = np.linalg.norm(f - As @ x)
        assert res <= tol * np.linalg.norm(p.sub_apply_P(s, f)) * (1 + 1e-8)


# -- Krylov solvers ------------------------------------------------------------------------------
def _krylov_min_residual(Aop, b, k):
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


def test_inner_gmres_is_krylov_minimiser(oracle_mod):
    p, w = _problem(oracle_mod, N=10, k=7.0, S=2, overlap=1)
    s = 3
    n = p.sub_n(s)
    assert n <= 64
    As = p.sub_A(s).toarray()
    P = np.column_stack([p.sub_apply_P(s, np.eye(n, dtype=complex)[:, c]) for c in range(n)])
    f = W.random_complex(n, 22)
    for k in (1, 3, 6):
        x, its = p.sub_solve(s, f, tol=1e-30, restart=40, maxit=k)
        assert its == k
        got = np.linalg.norm(f - As @ x)
        assert got == pytest.approx(_krylov_min_residual(P @ As, P @ f, k), rel=1e-8,
                                    abs=1e-13 * np.linalg.norm(f))


def test_fgmres_is_krylov_minimiser_with_exact_ras(oracle_mod):
    p, w = _problem(oracle_mod, N=8, k=6.0, S=2, overlap=1, exact=True)
    n = p.n
    A = p.matrix("A").toarray()
    Mi = np.column_stack([p.ras_apply(np.eye(n, dtype=complex)[:, c], inner_tol=0.0)[0]
                          for c in range(n)])
    f = W.random_complex(n, 4)
    for k in (1, 3, 6):
        x, st = p.solve(f, outer_tol=1e-30, outer_restart=50, outer_maxit=k, inner_tol=0.0,
                        raise_on_error=False)
        assert st["outer_its"] == k
        assert np.linalg.norm(f - A @ x) == pytest.approx(_krylov_min_residual(A @ Mi, f, k), rel=1e-8)


def test_one_subdomain_exact_is_one_iteration(oracle_mod):
    p = oracle_mod.Problem(20, 10.0, bc=1)
    p.setup_dd(1, 1, 1, [0, 20], [0, 20])
    p.setup_deflation()
    p.setup_exact()
    f = p.rhs(W.RHSSpec([W.PointSource(0.5, 0.5)]))
    x, st = p.solve(f, inner_tol=0.0)
    assert st["outer_its"] == 1


def test_solve_matches_direct_energy_identity_and_symmetry(oracle_mod):
    """k = 20, N = 32, 2x2 subdomains, overlap 2, centred point source, impedance boundary."""
    import scipy.sparse.linalg as spla
    N, k = 32, 20.0
    p, w = _problem(oracle_mod, N=N, k=k, S=2, overlap=2)
    f = p.rhs(w.rhs[0])
    x, st = p.solve(f, outer_tol=1e-10, inner_tol=1e-2)
    A = p.matrix("A")
    xd = spla.spsolve(A.tocsc(), f)
    assert np.linalg.norm(f - A @ x) <= 1e-10 * np.linalg.norm(f) * (1 + 1e-6)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert np.linalg.norm(x.imag) > 0.1 * np.linalg.norm(x)     # radiating: genuinely complex
    # Im(uᴴ A u) = -k uᴴ B u and uᴴ A u = uᴴ f: the power radiated through the boundary
    B = p.matrix("B")
    flux = np.vdot(xd, B @ xd).real
    assert flux > 0
    assert np.vdot(xd, f).imag == pytest.approx(-k * flux, rel=1e-9)
    # the SW-NE split is invariant under (i, j) -> (N-i, N-j) and (i, j) -> (j, i)
    U = xd.reshape(N + 1, N + 1)
    assert np.allclose(U, U[::-1, ::-1], rtol=0, atol=1e-10 * np.abs(U).max())
    assert np.allclose(U, U.T, rtol=0, atol=1e-10 * np.abs(U).max())
    assert st["outer_its"] < 40


def test_tight_inner_reproduces_direct_ras_history(oracle_mod):
    """Inner GMRES to 1e-13 gives the outer residual history of exact (LU) subdomain solves."""
    p, w = _problem(oracle_mod, N=40, k=16.0, S=2, overlap=2, exact=True)
    f = p.rhs(w.rhs[0])
    _, st_lu = p.solve(f, inner_tol=0.0)
    _, st_it = p.solve(f, inner_tol=1e-13)
    n = min(20, len(st_lu["res_history"]))
    h1, h2 = st_lu["res_history"][:n], st_it["res_history"][:n]
    assert np.max(np.abs(h1 - h2) / h1) < 1e-8
    assert st_lu["outer_its"] == st_it["outer_its"]
