"""Status paths of the C ABI on the GPU, reached through inputs made on the host (nothing here
faults, traps or hangs a GPU).

* Singular factors (§2: the paper assumes every subdomain problem is well posed).  For a finite
  wavenumber the P1 stencil's neighbour coefficient -1 - k²h²/12 never vanishes, so no valid
  box has a column without a non-zero pivot candidate; the one input that leaves none is a
  wavenumber whose k²h² overflows to infinity (k = 1e200 is finite, k² is not).  Every entry of
  E_j and A_j is then -inf, the device LU finds no finite pivot in column 0, and set-up returns
  HDD_ERR_SINGULAR_COARSE (hdd_setup_deflation) or HDD_ERR_SINGULAR_LOCAL (hdd_setup_exact)
  instead of producing NaN.
* Malformed decompositions: interfaces that do not run from 0 to N, gaps below two cells, and a
  box wider than the 256 nodes the local kernels stage are refused with HDD_ERR_INVALID_ARG.
* After each error the same context is reused for a valid problem, which then solves normally.
"""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ERR_INVALID_ARG, ERR_STATE, ERR_SINGULAR_COARSE, ERR_SINGULAR_LOCAL = 1, 2, 5, 6


def _solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2103_17081_gb300 import Solver
    return Solver(0)


def _valid_solve(s):
    w = W.make("tiny")
    s.assemble(w.k, w.N).setup_dd(w.Sx, w.Sy, w.overlap).setup_deflation()
    x, st = s.solve(s.build_rhs(w.rhs[0]), inner_prec=128)
    assert st["status_code"] == 0 and st["rel_res_true"] <= 1.0001e-6
    return st


def test_overflowing_wavenumber_reports_singular_factors():
    from paper_2103_17081_gb300 import HDDError
    s = _solver()
    s.assemble(1e200, 32).setup_dd(2, 2, 2)
    with pytest.raises(HDDError) as e:
        s.setup_deflation()
    assert e.value.code == ERR_SINGULAR_COARSE and "SINGULAR_COARSE" in str(e.value)
    with pytest.raises(HDDError) as e:
        s.setup_exact()
    assert e.value.code == ERR_SINGULAR_LOCAL and "SINGULAR_LOCAL" in str(e.value)
    # no factor was kept: a solve is refused, then the context takes a valid problem
    with pytest.raises(HDDError) as e:
        s.solve(s.build_rhs(W.RHSSpec([W.PointSource(0.5, 0.5)])))
    assert e.value.code == ERR_STATE
    _valid_solve(s)


@pytest.mark.parametrize("ifx,N,S", [([0, 10, 20, 31], 32, 3),     # does not end at N
                                     ([1, 10, 20, 32], 32, 3),     # does not start at 0
                                     ([0, 16, 17, 32], 32, 3),     # a gap of one cell
                                     ([0, 20, 10, 32], 32, 3),     # not increasing
                                     (None, 600, 2)])              # boxes 301 nodes wide
def test_malformed_decomposition_is_refused(ifx, N, S):
    from paper_2103_17081_gb300 import HDDError
    s = _solver()
    s.assemble(20.0, N)
    with pytest.raises(HDDError) as e:
        s.setup_dd(S, S, 2, ifx=ifx, ify=ifx)
    assert e.value.code == ERR_INVALID_ARG
    _valid_solve(s)
