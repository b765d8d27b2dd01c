"""Learned warm start: training-data recording, parameter initialisation, training loop and
checkpoints for the network behind hdd_cnn_* (include/hdd.h).

Orchestration only: every forward/backward pass, loss and Adam step runs in the library's
kernels; this module chooses the batches and reads/writes parameter files.

Training inputs are the right-hand sides the local solves actually see: the restricted outer
Krylov vectors R_j v of solves of seeded point-source / Gaussian-bump problems (the method's own
subdomain problems).  One batch = every subdomain image of one restricted vector.
"""
from __future__ import annotations

import struct
import zlib

import numpy as np

MAGIC = b"HDDCNN01"


def init_params(n_params: int, seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, last layer scaled by 0.1 so the
    initial guess is close to zero."""
    from .solver import Solver  # noqa: F401  (layer table lives with the library)
    layers = [(4, 32), (32, 32), (32, 32), (32, 2)]
    rng = np.random.default_rng(seed)
    out = []
    for l, (cin, cout) in enumerate(layers):
        std = np.sqrt(2.0 / (9 * cin)) * (0.1 if l == 3 else 1.0)
        w = rng.standard_normal(cout * 9 * cin) * std
        if cin == 4:                       # fourth input channel is always zero
            w.reshape(cout, 9, cin)[..., 3] = 0.0
        out.append(w)
        out.append(np.zeros(cout))
    p = np.concatenate(out).astype(np.float32)
    if p.size != n_params:
        raise ValueError("parameter layout mismatch")
    return p


def record_inputs(solver, specs, outer_its: int = 160, every: int = 4, **solve_kw):
    """Restricted outer Krylov vectors of partial solves, as packed complex128 tensors."""
    batches = []
    for spec in specs:
        f = solver.build_rhs(spec)
        kw = dict(outer_maxit=outer_its, outer_restart=outer_its, raise_on_error=False)
        kw.update(solve_kw)
        _, st = solver.solve(f, **kw)
        for j in range(0, st["outer_its"], every):
            batches.append(solver.local_op("R", solver.outer_vector(j)))
    return batches


def train(solver, batches, epochs: int = 4, lr: float = 1e-3, seed: int = 0, log=None):
    """Adam over the batches (shuffled each epoch); returns the per-epoch mean losses."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(batches))
        losses = [solver.cnn_train_step(batches[i], lr) for i in order]
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


def save(path: str, params: np.ndarray) -> None:
    """Parameter file: magic, count (u32), CRC32 of the FP32 payload (u32), payload."""
    a = np.ascontiguousarray(params, dtype=np.float32)
    payload = a.tobytes()
    with open(path, "wb") as fh:
        fh.write(MAGIC + struct.pack("<II", a.size, zlib.crc32(payload)) + payload)


def load(path: str) -> np.ndarray:
    with open(path, "rb") as fh:
        data = fh.read()
    if data[:8] != MAGIC:
        raise ValueError("not a warm-start parameter file")
    n, crc = struct.unpack("<II", data[8:16])
    payload = data[16:]
    if len(payload) != 4 * n or zlib.crc32(payload) != crc:
        raise ValueError("corrupt warm-start parameter file")
    return np.frombuffer(payload, dtype=np.float32).copy()


def _main(argv=None):
    """Command line: train a network on a workload and save it, time the inference, or compare
    warm- and zero-started solves of a held-out right-hand side."""
    import argparse
    import time

    import torch

    import workloads as W
    from .solver import Solver

    ap = argparse.ArgumentParser(prog="python -m paper_2103_17081_gb300.warmstart")
    ap.add_argument("command", choices=["train", "infer", "compare"])
    ap.add_argument("--workload", default="k200")
    ap.add_argument("--params", default=None, help="parameter file (read by infer/compare, written by train)")
    ap.add_argument("--seeds", type=int, default=8, help="training right-hand sides (seeds 100, 101, ...)")
    ap.add_argument("--outer-its", type=int, default=1270, help="outer iterations recorded per training solve")
    ap.add_argument("--every", type=int, default=32, help="record every n-th outer Krylov vector")
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--seed", type=int, default=1000, help="held-out right-hand side of compare")
    a = ap.parse_args(argv)
    w = W.make(a.workload)
    s = Solver.from_workload(w)
    if a.command == "train":
        s.cnn_set_params(init_params(s.cnn_num_params(), 0))
        specs = [W.make(a.workload, seed=100 + i).rhs[0] for i in range(a.seeds)]
        data = record_inputs(s, specs, outer_its=a.outer_its, every=a.every)
        hist = train(s, data, epochs=a.epochs, lr=a.lr, log=print)
        if a.params:
            save(a.params, s.cnn_get_params())
        print({"batches": len(data), "loss": hist})
        return 0
    s.cnn_set_params(load(a.params) if a.params else init_params(s.cnn_num_params(), 0))
    f = s.build_rhs(W.make(a.workload, seed=a.seed).rhs[0])
    if a.command == "infer":
        v = s.local_op("R", f / torch.linalg.vector_norm(f))
        out = {}
        for name, fn in (("tensor_core", s.cnn_infer), ("fp32_cuda_core", s.cnn_forward)):
            fn(v)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(a.reps):
                fn(v)
            e1.record()
            torch.cuda.synchronize()
            out[name + "_us"] = round(e0.elapsed_time(e1) * 1e3 / a.reps, 1)
        print(out)
        return 0
    res = {}
    for warm in (0, 1):
        s.solve(f, warm_start=warm)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, st = s.solve(f, warm_start=warm)
        torch.cuda.synchronize()
        res["warm" if warm else "zero"] = {"s": round(time.perf_counter() - t, 3), "outer": st["outer_its"],
                                           "inner_avg": round(st["inner_its_avg"], 3),
                                           "rel_res": st["rel_res_true"]}
    print(res)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(_main())
