"""GPU parity of the learned warm start: forward pass and gradients of the library's network
kernels against the numpy FP64 oracle (oracle/cnn.py, with the same BF16-rounded weights), and
training reducing the loss.  Tolerances: FP32 arithmetic (with the deflation projection applied
in FP32 around FP64 coarse solves) against FP64 — 1e-4 relative on the guess and on the loss,
1e-3 on the gradient vector."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import oracle
    from oracle import cnn
    from paper_2103_17081_gb300 import Solver
    from paper_2103_17081_gb300.warmstart import init_params
    w = W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45], name="ragged2")
    s = Solver.from_workload(w)
    p = oracle.from_workload(w)
    params = init_params(s.cnn_num_params(), seed=3)
    params[cnn.offsets()[3]:] *= 10.0                  # a non-trivial output layer
    s.cnn_set_params(params)
    fo, _ = s.offsets()
    f = W.random_complex_fast(fo[-1], 9)
    from test_oracle_cnn import projections
    batch = [(f[fo[t]:fo[t + 1]], (p.box(t)["ny"], p.box(t)["nx"]), p.sub_A(t)) + projections(p, t)
             for t in range(p.nsub)]
    kh = w.k / w.N
    return torch, s, p, cnn, cnn.bf16_round(params), f, fo, batch, kh


def test_forward_matches_oracle():
    torch, s, p, cnn, pb, f, fo, batch, kh = _setup()
    x0 = s.cnn_forward(torch.from_numpy(f).cuda()).cpu().numpy()
    for t, (ft, shape, *_) in enumerate(batch):
        ref = cnn.guess(pb, ft, shape, kh)
        got = x0[fo[t]:fo[t + 1]]
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), t


def test_loss_and_gradient_match_oracle():
    torch, s, p, cnn, pb, f, fo, batch, kh = _setup()
    L, g = s.cnn_loss_grad(torch.from_numpy(f).cuda())
    Lr, gr = cnn.loss_and_grad(pb, batch, kh)
    assert L == pytest.approx(Lr, rel=1e-4)
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    off = cnn.offsets()
    for l in range(4):                                   # every layer, not just the largest
        a, b = g[off[l]:off[l + 1]], gr[off[l]:off[l + 1]]
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b), l


def test_training_reduces_loss():
    torch, s, p, cnn, pb, f, fo, batch, kh = _setup()
    from paper_2103_17081_gb300 import warmstart
    s.cnn_set_params(warmstart.init_params(s.cnn_num_params(), seed=0))
    w = W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45])
    data = warmstart.record_inputs(s, [W.RHSSpec([W.PointSource(0.4, 0.6)])], outer_its=24, every=2)
    assert len(data) >= 10
    L0 = np.mean([s.cnn_loss_grad(d, with_grad=False)[0] for d in data])
    warmstart.train(s, data, epochs=6, lr=2e-3)
    L1 = np.mean([s.cnn_loss_grad(d, with_grad=False)[0] for d in data])
    assert L1 < 0.9 * L0
    # the checkpoint round-trips exactly
    import os
    import tempfile
    path = os.path.join(tempfile.mkdtemp(), "ws.bin")
    prm = s.cnn_get_params()
    warmstart.save(path, prm)
    assert np.array_equal(warmstart.load(path), prm)
