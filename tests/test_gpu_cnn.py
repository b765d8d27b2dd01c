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
    # the C ABI reads and writes the same format (and rejects a corrupted file)
    s.cnn_set_params(warmstart.init_params(s.cnn_num_params(), seed=7))
    s.cnn_load(path)
    assert np.array_equal(s.cnn_get_params(), prm)
    path2 = path + ".c"
    s.cnn_save(path2)
    assert open(path2, "rb").read() == open(path, "rb").read()
    raw = bytearray(open(path, "rb").read())
    raw[40] ^= 1
    open(path2, "wb").write(bytes(raw))
    from paper_2103_17081_gb300 import HDDError
    with pytest.raises(HDDError):
        s.cnn_load(path2)


def test_tensor_core_inference_matches_oracle():
    """hdd_cnn_infer (layers 2-4 on tcgen05, BF16 activations) against the oracle forward with
    BF16-rounded activations, on boxes of six different widths (frames of 2-3 tiles of 128
    positions, so first, interior and ragged last tiles all occur)."""
    torch, s, p, cnn, pb, f, fo, batch, kh = _setup()
    x0 = s.cnn_infer(torch.from_numpy(f).cuda()).cpu().numpy()
    for t, (ft, shape, *_) in enumerate(batch):
        ref = cnn.guess(pb, ft, shape, kh, act_bf16=True)
        got = x0[fo[t]:fo[t + 1]]
        assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref), t


def test_warm_start_gain_k100():
    """What the trained network gains: a network trained on the restricted outer Krylov vectors of
    four seeded k=100 solves (N=320, 4x4 subdomains) lowers the total inner iteration count of
    RAS applications to 20 outer Krylov vectors of a held-out right-hand side (another seed), and
    with it a whole solve still meets the outer tolerance, within +10 % outer iterations, with the
    zero-guess method's solution.  (The per-solve average moves by only a few percent at this size,
    so the gain is measured over the preconditioner applications, where it is systematic.)
    Inference is the tensor-core path, checked against the oracle at this box size (81 and 83
    nodes wide)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import oracle
    from oracle import cnn
    from paper_2103_17081_gb300 import Solver, warmstart
    w = W.make("k100")
    s = Solver.from_workload(w)
    s.cnn_set_params(warmstart.init_params(s.cnn_num_params(), seed=0))
    specs = [W.make("k100", seed=100 + i).rhs[0] for i in range(4)]
    data = warmstart.record_inputs(s, specs, outer_its=400, every=8)
    hist = warmstart.train(s, data, epochs=4, lr=1e-3)
    assert hist[-1] < 0.2
    # tensor-core inference on two full-size boxes against the oracle (BF16 activations)
    p = oracle.from_workload(w)
    pb = cnn.bf16_round(s.cnn_get_params())
    fo, _ = s.offsets()
    fv = data[-1]
    x0 = s.cnn_infer(fv).cpu().numpy()
    fh = fv.cpu().numpy()
    for t in (0, 5):
        b = p.box(t)
        ref = cnn.guess(pb, fh[fo[t]:fo[t + 1]], (b["ny"], b["nx"]), w.k / w.N, act_bf16=True)
        assert np.linalg.norm(x0[fo[t]:fo[t + 1]] - ref) <= 2e-3 * np.linalg.norm(ref), t
    f = s.build_rhs(W.make("k100", seed=1000).rhs[0])
    s.solve(f, warm_start=0, outer_maxit=200, outer_restart=200, raise_on_error=False)
    vs = [s.outer_vector(j).clone() for j in range(0, 200, 10)]
    cold = sum(sum(s.ras_apply(v, inner_tol=1e-2, inner_prec=64, warm_start=0)[1]) for v in vs)
    warm = sum(sum(s.ras_apply(v, inner_tol=1e-2, inner_prec=64, warm_start=1)[1]) for v in vs)
    assert warm < cold, (warm, cold)
    xc, stc = s.solve(f, warm_start=0)
    xw, stw = s.solve(f, warm_start=1)
    assert stw["rel_res_true"] <= 1e-6 * 1.0001
    assert stw["outer_its"] <= 1.1 * stc["outer_its"]
    # same solution: two different iterates at residual 1e-6 may differ by ~cond·1e-6, so the
    # solutions are compared at outer tolerance 1e-8
    xc, _ = s.solve(f, warm_start=0, outer_tol=1e-8)
    xw, _ = s.solve(f, warm_start=1, outer_tol=1e-8)
    assert float(torch.linalg.vector_norm(xw - xc) / torch.linalg.vector_norm(xc)) < 1e-6


def test_batched_inference_matches_single_rhs():
    """Tensor-core inference over the tasks of two batched right-hand sides gives, for each RHS,
    the single-RHS result (tile tables and padded frames span all tasks)."""
    torch, s, p, cnn, pb, f, fo, batch, kh = _setup()
    from paper_2103_17081_gb300 import Solver
    w = W.custom(17.0, 45, 3, 2, Sy=4, ifx=[0, 11, 29, 45], name="ragged2")
    sb = Solver.from_workload(w).setup_batch(2)
    sb.cnn_set_params(s.cnn_get_params())
    n1 = fo[-1]
    f2 = np.concatenate([f, W.random_complex_fast(n1, 10)])
    xb = sb.cnn_infer(torch.from_numpy(f2).cuda()).cpu().numpy()
    x0 = s.cnn_infer(torch.from_numpy(f2[:n1]).cuda()).cpu().numpy()
    x1 = s.cnn_infer(torch.from_numpy(f2[n1:]).cuda()).cpu().numpy()
    assert np.array_equal(xb[:n1], x0) and np.array_equal(xb[n1:], x1)
