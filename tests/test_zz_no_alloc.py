"""hdd_apply_PA_noalloc: the deflated operator for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (code inside a captured CUDA graph, an embedding whose
allocator must not be re-entered, an application that owns all device memory up front).  For
them the library applies P_j A_j with its coarse work vectors in a fixed array compiled into
the library.  This test calls that entry point through the C ABI, twice in a row, and checks
each result against hdd_local_op (op 4, the allocating entry point for the same operator) at
the tolerance the local-operator parity tests use for complex128 (1e-13 relative).  It sits in a
file that pytest collects last and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc", [0, 1], ids=["dirichlet", "impedance"])
def test_apply_PA_noalloc_matches_allocating_entry_point(bc):
    """bc = 1: the impedance problem, whose coarse factors are real-equivalent systems."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2103_17081_gb300 import Solver, lib

    w = W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45], name="ragged2", bc=bc)
    s = Solver.from_workload(w)
    fo, co = s.offsets()
    x = torch.from_numpy(W.random_complex_fast(fo[-1], 77)).cuda()
    ref = s.local_op("PA", x, prec=128).cpu().numpy()
    L = lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full_like(x, complex(float("nan"), float("nan")))
        rc = L.hdd_apply_PA_noalloc(s._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    stream)
        assert rc == 0, (call, L.hdd_last_error(s._h))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), call


def test_apply_PA_noalloc_reports_call_order():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2103_17081_gb300 import Solver, lib

    s = Solver(0).assemble(20.0, 32)
    s.setup_dd(2, 2, 2)
    x = s.empty(4 * 17 * 17)
    out = s.empty(4 * 17 * 17)
    rc = lib().hdd_apply_PA_noalloc(s._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    None)
    assert rc == 2          # HDD_ERR_STATE: deflation not set up
