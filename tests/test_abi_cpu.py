"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports every entry
point declared in include/hdd.h; the product path refuses to run without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hdd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdd_[A-Za-z_]+)\s*\(", src)))


def test_header_matches_binding():
    from paper_2103_17081_gb300 import SYMBOLS
    assert sorted(SYMBOLS) == _declared()


def test_option_keys_match_binding_and_library():
    """Every HDD_OPT_* key include/hdd.h defines is in the binding's OPTIONS table under its
    lower-case name with the same value, and hdd_set_option handles it."""
    src = open(os.path.join(ROOT, "include", "hdd.h")).read()
    keys = {name.lower(): int(v) for name, v in re.findall(r"#define HDD_OPT_([A-Z0-9_]+)\s+(\d+)", src)}
    assert keys, "no option keys found in the header"
    from paper_2103_17081_gb300 import Solver
    assert Solver.OPTIONS == keys
    api = open(os.path.join(ROOT, "paper_2103_17081_gb300", "csrc", "hdd_api.cu")).read()
    for name in keys:
        assert re.search(r"key == HDD_OPT_%s\)" % name.upper(), api), name


def test_library_builds_and_exports_all_symbols():
    from paper_2103_17081_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hdd_[A-Za-z_]+)\b", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)            # loads without a GPU
    for s in _declared():
        assert hasattr(lib, s)


def test_status_strings_without_gpu():
    from paper_2103_17081_gb300 import lib
    L = lib()
    assert L.hdd_status_str(0) == b"HDD_OK"
    assert L.hdd_status_str(5) == b"HDD_ERR_SINGULAR_COARSE"
    # no device here: creating a context must fail with a status, not crash
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert L.hdd_create(ctypes.byref(h), 0) != 0
        assert L.hdd_last_error(None) == b""


def test_solver_needs_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2103_17081_gb300 import Solver
    with pytest.raises(RuntimeError):
        Solver(0)


def test_oracle_and_product_share_no_code():
    """The oracle never imports the package and the package never imports the oracle."""
    for d, other in (("oracle", "paper_2103_17081_gb300"), ("paper_2103_17081_gb300", "oracle")):
        base = os.path.join(ROOT, d)
        for dp, _, files in os.walk(base):
            for fn in files:
                if fn.endswith((".py", ".c", ".h", ".cu", ".cuh")):
                    txt = open(os.path.join(dp, fn), encoding="utf-8").read()
                    assert not re.search(rf"^\s*(import|from)\s+{other}\b", txt, re.M), (fn, other)
                    assert f'#include "{other}' not in txt


def test_sweep_table_layout():
    """The paper-table sweep prints 'outer (avg inner)' per (ppwl, k) row and N column."""
    from paper_2103_17081_gb300.sweep import table
    rows = [{"ppwl": 10, "k": 20, "n_glob": 30, "N": 4, "inner": "1e-2", "outer_its": 21, "inner_avg": 5.0},
            {"ppwl": 10, "k": 20, "n_glob": 30, "N": 9, "inner": "1e-2", "outer_its": 30, "inner_avg": 6.25},
            {"ppwl": 10, "k": 20, "n_glob": 30, "N": 4, "inner": "LU", "outer_its": 20, "inner_avg": 0.0}]
    t = table(rows, "1e-2").splitlines()
    assert t[0] == "| ppwl | k | n_glob | N=4 | N=9 |"
    assert t[2] == "| 10 | 20 | 30 | 21 (5) | 30 (6.25) |"
    assert table(rows, "LU").splitlines()[2] == "| 10 | 20 | 30 | 20 |"


@pytest.mark.parametrize("diag", [0, 1])
def test_impedance_stencil_rows_match_oracle_assembly(oracle_mod, diag):
    """The node-class rows every kernel applies under the impedance condition (host-only
    hdd_stencil_rows) equal the rows of the oracle's element-by-element assembly of A and M at
    every node of the mesh; slots towards nodes outside the square are zero."""
    import numpy as np
    from paper_2103_17081_gb300 import lib
    L = lib()
    offs = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)] + ([(1, 1), (-1, -1)] if diag == 0 else [(1, -1), (-1, 1)])
    for (N, k) in [(6, 3.0), (9, 7.5), (16, 20.0)]:
        coef = np.zeros(2 * 63)
        mass = np.zeros(63)
        assert L.hdd_stencil_rows(N, k, diag, coef.ctypes.data_as(ctypes.c_void_p),
                                  mass.ctypes.data_as(ctypes.c_void_p)) == 0
        coef = (coef[0::2] + 1j * coef[1::2]).reshape(9, 7)
        mass = mass.reshape(9, 7)
        p = oracle_mod.Problem(N, k, diag=diag, bc=1)
        A, M = p.matrix("A").toarray(), p.matrix("M").toarray()
        for j in range(N + 1):
            for i in range(N + 1):
                cls = (0 if i == 0 else (2 if i == N else 1)) + 3 * (0 if j == 0 else (2 if j == N else 1))
                r = p.node_index(i, j)
                cols = [p.node_index(i + dx, j + dy) for dx, dy in offs]
                ra = np.array([A[r, c] if c >= 0 else 0.0 for c in cols])
                rm = np.array([M[r, c] if c >= 0 else 0.0 for c in cols])
                assert np.count_nonzero(A[r]) == np.count_nonzero(ra)     # no coupling outside the slots
                assert np.allclose(coef[cls], ra, rtol=1e-14, atol=1e-14 * np.abs(ra).max())
                assert np.allclose(mass[cls], rm, rtol=1e-14, atol=1e-14 * np.abs(rm).max())
                for q, c in enumerate(cols):
                    if c < 0:
                        assert coef[cls, q] == 0 and mass[cls, q] == 0
    bad = np.zeros(2 * 63)
    assert L.hdd_stencil_rows(3, 1.0, 0, bad.ctypes.data_as(ctypes.c_void_p), None) != 0
    assert L.hdd_stencil_rows(8, 1.0, 2, bad.ctypes.data_as(ctypes.c_void_p), None) != 0


@pytest.mark.parametrize("bc", [0, 1])
def test_sweep_settings_follow_the_paper_recipe(oracle_mod, bc):
    """Every sweep setting has n_glob = 1.5k (10 ppwl) or 3k (20 ppwl) intervals, S x S uniform
    subdomains, one layer of overlap, a centred point source and the chosen boundary condition;
    the oracle accepts the decomposition."""
    from paper_2103_17081_gb300.sweep import settings
    st = settings([20, 40], [10, 20], [2, 3], bc=bc)
    assert len(st) == 8
    for (ppwl, k, n_glob, S, w) in st:
        assert n_glob == round(k * (1.5 if ppwl == 10 else 3.0)) and w.N == n_glob
        assert (w.Sx, w.Sy, w.overlap, w.bc) == (S, S, 1, bc)
        assert [(q.x, q.y) for q in w.rhs[0].points] == [(0.5, 0.5)]
    ppwl, k, n_glob, S, w = st[1]
    p = oracle_mod.Problem(w.N, w.k, bc=w.bc)
    p.setup_dd(w.Sx, w.Sy, w.overlap, w.ifx, w.ify)
    assert p.n == ((w.N + 1) ** 2 if bc else (w.N - 1) ** 2)
