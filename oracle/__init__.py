"""CPU oracle of the method — TEST INFRASTRUCTURE ONLY.

A plain, slow, complex128 implementation of the whole solver, written from the paper's
definitions: P1 assembly (Eq. 2), overlapping Cartesian decomposition and RAS (Eq. 3), two-level
deflation with the quadratic Bézier deflation matrix (Eq. 4, Eq. 5), deflated GMRES on each
subdomain and FGMRES outside (§3).  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import it; it shares no code with the CUDA path.

The compute lives in hdd_oracle.c (gcc, OpenMP across independent subdomain solves); this module
only marshals numpy arrays through ctypes.  Parity is pinned by tests/test_oracle_*.py against
closed forms, dense direct solves, invariants and brute force.  The paper's iteration tables are
trend context only ("parity unpinned" for the counts; see the test module headers).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OracleError(RuntimeError):
    pass


_ERR = {1: "bad argument", 2: "bad call order", 3: "singular pivot", 4: "no convergence",
        5: "non-finite value"}


class SolveParams(C.Structure):
    _fields_ = [("outer_tol", C.c_double), ("outer_restart", C.c_int), ("outer_maxit", C.c_int),
                ("inner_tol", C.c_double), ("inner_restart", C.c_int), ("inner_maxit", C.c_int),
                ("two_level", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("status", C.c_int), ("rel_res_true", C.c_double),
                ("inner_its_total", C.c_longlong), ("inner_its_avg", C.c_double),
                ("inner_its_max", C.c_int), ("inner_maxit_hits", C.c_longlong),
                ("n_history", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, I, D, Z = C.c_void_p, C.c_int, C.c_double, C.c_void_p
        L.or_create.restype = P
        L.or_create.argtypes = [I, D, I]
        L.or_create_bc.restype = P
        L.or_create_bc.argtypes = [I, D, I, I]
        L.or_destroy.argtypes = [P]
        for name in ("or_n", "or_nsub"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = I
        L.or_nnz.argtypes = [P, I]
        L.or_nnz.restype = I
        L.or_get_csr.argtypes = [P, I, Z, Z, Z]
        L.or_get_csr_imag.argtypes = [P, I, Z]
        L.or_apply_global.argtypes = [P, I, Z, Z]
        L.or_rhs_point.argtypes = [P, D, D, D, Z]
        L.or_rhs_gauss.argtypes = [P, D, D, D, D, Z]
        L.or_rhs_manufactured.argtypes = [P, Z]
        L.or_setup_dd.argtypes = [P, I, I, I, Z, Z]
        L.or_setup_dd.restype = I
        L.or_sub_box.argtypes = [P, I, Z]
        for name in ("or_sub_n", "or_sub_m"):
            getattr(L, name).argtypes = [P, I]
            getattr(L, name).restype = I
        L.or_sub_nnz.argtypes = [P, I, I]
        L.or_sub_nnz.restype = I
        L.or_sub_get_csr.argtypes = [P, I, I, Z, Z, Z]
        L.or_sub_get_csr_imag.argtypes = [P, I, I, Z]
        for name in ("or_sub_restrict", "or_sub_apply_A", "or_sub_apply_Z", "or_sub_apply_Zt",
                     "or_sub_apply_PA", "or_sub_apply_P"):
            getattr(L, name).argtypes = [P, I, Z, Z]
        L.or_setup_deflation.argtypes = [P]
        L.or_setup_deflation.restype = I
        L.or_setup_exact.argtypes = [P]
        L.or_setup_exact.restype = I
        L.or_sub_E_band.argtypes = [P, I, Z]
        L.or_sub_E_dense.argtypes = [P, I, Z]
        L.or_sub_E_dense_imag.argtypes = [P, I, Z]
        L.or_sub_coarse_solve.argtypes = [P, I, Z, Z]
        L.or_sub_coarse_solve.restype = I
        L.or_sub_solve.argtypes = [P, I, Z, Z, D, I, I, Z, C.POINTER(I)]
        L.or_sub_solve.restype = I
        L.or_sub_solve_exact.argtypes = [P, I, Z, Z]
        L.or_sub_solve_exact.restype = I
        L.or_ras_apply.argtypes = [P, Z, Z, D, I, I, C.POINTER(C.c_longlong), C.POINTER(I),
                                   C.POINTER(C.c_longlong)]
        L.or_ras_apply.restype = I
        L.or_solve.argtypes = [P, Z, Z, C.POINTER(SolveParams), C.POINTER(Stats), Z, I]
        L.or_solve.restype = I
        L.or_cgs2.argtypes = [Z, I, I, Z, Z]
        L.or_cgs2.restype = D
        L.or_band_lu.argtypes = [I, I, I, Z, Z]
        L.or_band_lu.restype = I
        L.or_band_solve.argtypes = [I, I, I, Z, Z, Z]
        L.or_band_lu_z.argtypes = [I, I, I, Z, Z]
        L.or_band_lu_z.restype = I
        L.or_band_solve_z.argtypes = [I, I, I, Z, Z, Z]
        L.or_set_threads.argtypes = [I]
        L.or_get_threads.restype = I
        L.or_setup_coarse_grid.argtypes = [P, I]
        L.or_setup_coarse_grid.restype = I
        L.or_cg_n.argtypes = [P]
        L.or_cg_n.restype = I
        for name in ("or_cg_apply_P", "or_cg_apply_Pt", "or_cg_solve"):
            getattr(L, name).argtypes = [P, Z, Z]
            getattr(L, name).restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what}: {_ERR.get(st, st)}")


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def cgs2(V: np.ndarray, w):
    """Outer CGS2 of the oracle: (w orthogonalised against the columns of V, coefficients h, ||w||).
    V is n x nv complex128; it is passed column-major without a copy when already Fortran-ordered."""
    V = np.asfortranarray(V, dtype=np.complex128)
    n, nv = V.shape
    w = _c128(w).copy()
    h = np.zeros(nv, dtype=np.complex128)
    r = lib().or_cgs2(_ptr(V), n, nv, _ptr(w), _ptr(h))
    return w, h, r


def band_lu(ab: np.ndarray, m: int, kl: int, ku: int):
    """In-place banded LU with partial pivoting of row-band storage (m x (2kl+ku+1))."""
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    piv = np.zeros(m, dtype=np.int32)
    st = lib().or_band_lu(m, kl, ku, _ptr(ab), _ptr(piv))
    _check(st, "band_lu")
    return ab, piv


def band_solve(ab, piv, m, kl, ku, b):
    x = _c128(b).copy()
    lib().or_band_solve(m, kl, ku, _ptr(np.ascontiguousarray(ab, dtype=np.float64)),
                        _ptr(np.ascontiguousarray(piv, dtype=np.int32)), _ptr(x))
    return x


def band_lu_z(ab: np.ndarray, m: int, kl: int, ku: int):
    """Complex banded LU with partial pivoting (largest modulus), same storage as band_lu."""
    ab = _c128(ab).copy()
    piv = np.zeros(m, dtype=np.int32)
    st = lib().or_band_lu_z(m, kl, ku, _ptr(ab), _ptr(piv))
    _check(st, "band_lu_z")
    return ab, piv


def band_solve_z(ab, piv, m, kl, ku, b):
    x = _c128(b).copy()
    lib().or_band_solve_z(m, kl, ku, _ptr(_c128(ab)), _ptr(np.ascontiguousarray(piv, dtype=np.int32)),
                          _ptr(x))
    return x


BC = {"dirichlet": 0, "sommerfeld": 1}
_WHICH = {"A": 0, "K": 1, "M": 2, "B": 3}


class Problem:
    """Discrete Helmholtz problem with its decomposition and local deflation (oracle side).

    bc 0: u = 0 on the boundary (Eq. 1), unknowns at the (N-1)² interior nodes.  bc 1: the
    first-order absorbing condition du/dn - i k u = 0 on all four sides, unknowns at all (N+1)²
    nodes, A = K - k²M - i k B complex symmetric (B the boundary mass matrix).
    """

    def __init__(self, N: int, k: float, diag: int = 0, bc: int = 0):
        self.N, self.k, self.diag, self.bc = int(N), float(k), int(diag), int(bc)
        self._h = lib().or_create_bc(self.N, self.k, self.diag, self.bc)
        if not self._h:
            raise OracleError("or_create failed")
        self.n = lib().or_n(self._h)
        self.nsub = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    # -- assembly ----------------------------------------------------------------------------
    def matrix(self, which: str = "A"):
        """CSR of A, K, M or B (B: boundary mass, empty for Dirichlet); complex where A is."""
        import scipy.sparse as sp
        w = _WHICH[which]
        nnz = lib().or_nnz(self._h, w)
        rp = np.zeros(self.n + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz, dtype=np.float64)
        lib().or_get_csr(self._h, w, _ptr(rp), _ptr(ci), _ptr(v))
        if self.bc and which == "A":
            vi = np.zeros(nnz, dtype=np.float64)
            lib().or_get_csr_imag(self._h, w, _ptr(vi))
            v = v + 1j * vi
        return sp.csr_matrix((v, ci, rp), shape=(self.n, self.n))

    def node_index(self, i: int, j: int) -> int:
        """Unknown index of mesh node (i, j) (x fastest), -1 if it is not an unknown."""
        lo, hi = (0, self.N) if self.bc else (1, self.N - 1)
        if not (lo <= i <= hi and lo <= j <= hi):
            return -1
        return (i - lo) + (j - lo) * (hi - lo + 1)

    def apply(self, x, which: str = "A"):
        x = _c128(x)
        y = np.empty_like(x)
        lib().or_apply_global(self._h, _WHICH[which], _ptr(x), _ptr(y))
        return y

    # -- right-hand sides ----------------------------------------------------------------------
    def rhs(self, spec) -> np.ndarray:
        """Load vector of a workloads.RHSSpec: point sources F = amp e_c, bumps F += M g_I."""
        f = np.zeros(self.n, dtype=np.complex128)
        for p in spec.points:
            lib().or_rhs_point(self._h, p.x, p.y, p.amp, _ptr(f))
        for b in spec.bumps:
            lib().or_rhs_gauss(self._h, b.cx, b.cy, b.sigma, b.amp, _ptr(f))
        return f

    def rhs_manufactured(self) -> np.ndarray:
        f = np.zeros(self.n, dtype=np.complex128)
        lib().or_rhs_manufactured(self._h, _ptr(f))
        return f

    # -- decomposition --------------------------------------------------------------------------
    def setup_dd(self, Sx: int, Sy: int, overlap: int, ifx, ify):
        ifx = np.ascontiguousarray(ifx, dtype=np.int32)
        ify = np.ascontiguousarray(ify, dtype=np.int32)
        _check(lib().or_setup_dd(self._h, Sx, Sy, overlap, _ptr(ifx), _ptr(ify)), "setup_dd")
        self.nsub = lib().or_nsub(self._h)

    def box(self, s: int) -> dict:
        b = np.zeros(8, dtype=np.int32)
        lib().or_sub_box(self._h, s, _ptr(b))
        keys = ("ix0", "ix1", "iy0", "iy1", "ox0", "ox1", "oy0", "oy1")
        d = {k: int(v) for k, v in zip(keys, b)}
        d["nx"] = d["ix1"] - d["ix0"] + 1
        d["ny"] = d["iy1"] - d["iy0"] + 1
        return d

    def sub_n(self, s: int) -> int:
        return lib().or_sub_n(self._h, s)

    def sub_m(self, s: int) -> int:
        return lib().or_sub_m(self._h, s)

    def restrict(self, s: int, v) -> np.ndarray:
        v = _c128(v)
        out = np.empty(self.sub_n(s), dtype=np.complex128)
        lib().or_sub_restrict(self._h, s, _ptr(v), _ptr(out))
        return out

    def _sub_csr(self, s: int, which: int, shape):
        import scipy.sparse as sp
        nnz = lib().or_sub_nnz(self._h, s, which)
        rp = np.zeros(shape[0] + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz, dtype=np.float64)
        lib().or_sub_get_csr(self._h, s, which, _ptr(rp), _ptr(ci), _ptr(v))
        if self.bc and which == 0:
            vi = np.zeros(nnz, dtype=np.float64)
            lib().or_sub_get_csr_imag(self._h, s, which, _ptr(vi))
            v = v + 1j * vi
        return sp.csr_matrix((v, ci, rp), shape=shape)

    def sub_A(self, s: int):
        n = self.sub_n(s)
        return self._sub_csr(s, 0, (n, n))

    def sub_Z(self, s: int):
        return self._sub_csr(s, 1, (self.sub_n(s), self.sub_m(s)))

    def _sub_op(self, fn, s, v, nout):
        v = _c128(v)
        out = np.empty(nout, dtype=np.complex128)
        getattr(lib(), fn)(self._h, s, _ptr(v), _ptr(out))
        return out

    def sub_apply_A(self, s, v):
        return self._sub_op("or_sub_apply_A", s, v, self.sub_n(s))

    def sub_apply_Z(self, s, c):
        return self._sub_op("or_sub_apply_Z", s, c, self.sub_n(s))

    def sub_apply_Zt(self, s, f):
        return self._sub_op("or_sub_apply_Zt", s, f, self.sub_m(s))

    def sub_apply_PA(self, s, v):
        return self._sub_op("or_sub_apply_PA", s, v, self.sub_n(s))

    def sub_apply_P(self, s, v):
        return self._sub_op("or_sub_apply_P", s, v, self.sub_n(s))

    # -- deflation ---------------------------------------------------------------------------------
    def setup_deflation(self):
        _check(lib().or_setup_deflation(self._h), "setup_deflation")

    def setup_exact(self):
        _check(lib().or_setup_exact(self._h), "setup_exact")

    def E_band(self, s: int):
        b = np.zeros(2, dtype=np.int32)
        lib().or_sub_E_band(self._h, s, _ptr(b))
        return int(b[0]), int(b[1])

    def E_dense(self, s: int) -> np.ndarray:
        m = self.sub_m(s)
        if m > 400:
            raise OracleError("dense E is kept only for m <= 400")
        E = np.zeros((m, m), dtype=np.float64)
        lib().or_sub_E_dense(self._h, s, _ptr(E))
        if self.bc:
            Ei = np.zeros((m, m), dtype=np.float64)
            lib().or_sub_E_dense_imag(self._h, s, _ptr(Ei))
            return E + 1j * Ei
        return E

    def coarse_solve(self, s: int, y) -> np.ndarray:
        y = _c128(y)
        x = np.empty_like(y)
        _check(lib().or_sub_coarse_solve(self._h, s, _ptr(y), _ptr(x)), "coarse_solve")
        return x

    def sub_solve(self, s: int, f, tol: float, restart: int = 30, maxit: int = 1000, x0=None):
        f = _c128(f)
        x = np.empty_like(f)
        its = C.c_int(0)
        x0p = _ptr(_c128(x0)) if x0 is not None else None
        keep = _c128(x0) if x0 is not None else None
        if keep is not None:
            x0p = _ptr(keep)
        _check(lib().or_sub_solve(self._h, s, _ptr(f), x0p, tol, restart, maxit, _ptr(x),
                                  C.byref(its)), "sub_solve")
        return x, its.value

    def sub_solve_exact(self, s: int, f) -> np.ndarray:
        f = _c128(f)
        x = np.empty_like(f)
        _check(lib().or_sub_solve_exact(self._h, s, _ptr(f), _ptr(x)), "sub_solve_exact")
        return x

    # -- RAS and outer solve -----------------------------------------------------------------------
    def ras_apply(self, v, inner_tol: float, inner_restart: int = 30, inner_maxit: int = 1000):
        v = _c128(v)
        z = np.zeros_like(v)
        tot, mx, hits = C.c_longlong(0), C.c_int(0), C.c_longlong(0)
        _check(lib().or_ras_apply(self._h, _ptr(v), _ptr(z), inner_tol, inner_restart,
                                  inner_maxit, C.byref(tot), C.byref(mx), C.byref(hits)),
               "ras_apply")
        return z, {"inner_its_total": tot.value, "inner_its_max": mx.value,
                   "inner_maxit_hits": hits.value}

    # -- two-level variant: grid coarse space ------------------------------------------------
    def setup_coarse_grid(self, c: int = 2):
        """P1 on the mesh of N/c intervals: interpolation P, lumped coarse operator A_H, factored."""
        _check(lib().or_setup_coarse_grid(self._h, int(c)), "setup_coarse_grid")

    def cg_n(self) -> int:
        return lib().or_cg_n(self._h)

    def cg_P(self, uH):
        uH = _c128(uH)
        u = np.empty(self.n, dtype=np.complex128)
        lib().or_cg_apply_P(self._h, _ptr(uH), _ptr(u))
        return u

    def cg_Pt(self, v):
        v = _c128(v)
        vH = np.empty(self.cg_n(), dtype=np.complex128)
        lib().or_cg_apply_Pt(self._h, _ptr(v), _ptr(vH))
        return vH

    def cg_solve(self, yH):
        yH = _c128(yH)
        xH = np.empty_like(yH)
        lib().or_cg_solve(self._h, _ptr(yH), _ptr(xH))
        return xH

    def solve(self, f, outer_tol=1e-6, outer_restart=2000, outer_maxit=2000, inner_tol=1e-2,
              inner_restart=30, inner_maxit=1000, raise_on_error=True, two_level=0):
        f = _c128(f)
        x = np.zeros_like(f)
        prm = SolveParams(outer_tol, outer_restart, outer_maxit, inner_tol, inner_restart,
                          inner_maxit, int(bool(two_level)))
        st = Stats()
        hist = np.zeros(outer_maxit + 1, dtype=np.float64)
        rc = lib().or_solve(self._h, _ptr(f), _ptr(x), C.byref(prm), C.byref(st), _ptr(hist),
                            len(hist))
        stats = {k: getattr(st, k) for k, _ in Stats._fields_}
        stats["res_history"] = hist[: st.n_history].copy()
        if rc != 0 and raise_on_error:
            raise OracleError(f"solve: {_ERR.get(rc, rc)} after {st.outer_its} its "
                              f"(rel res {st.rel_res_true:.3e})")
        return x, stats


def from_workload(w, deflation: bool = True, exact: bool = False) -> Problem:
    """Assemble a workloads.Workload on the oracle side and set up its decomposition."""
    p = Problem(w.N, w.k, bc=getattr(w, "bc", 0))
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    if deflation:
        p.setup_deflation()
    if exact:
        p.setup_exact()
    return p
