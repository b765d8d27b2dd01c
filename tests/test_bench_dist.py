"""Multi-process paths of bench.py on the CPU (gloo, two ranks): the step time is the maximum over
the replicas on every rank, and the reference arm prints only on rank 0."""
import contextlib
import io
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_max_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(port, out), nprocs=2, join=True)
        assert out[0] == 2.5 and out[1] == 2.5


def test_max_over_ranks_without_a_group():
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1",
                                     "--warmup", "0"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.main() == 0
    assert buf.getvalue() == ""


def test_reference_arm_json_line_keys(monkeypatch):
    """The reference arm (CPU oracle, bounded sample) prints one JSON line with the contract's
    keys, the same workload keys as the GPU arm, and a cpu_baseline / e2e of its own."""
    import json

    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1",
                                     "--warmup", "0"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.main() == 0
    lines = [ln for ln in buf.getvalue().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert set(bench.workload_config(bench.W.make("tiny"))) <= set(d["config"])
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_oracle_estimate_recovers_a_cost_model(monkeypatch):
    """With iteration i costing r (a third of it during a 50-iteration start-up) plus c·(i+1)
    for its CGS2, the estimate from samples of 100, 200 and 400 iterations reproduces the exact
    total for J iterations; the former two-sample quadratic fit did not (it read the cheap
    start-up as growth)."""
    import bench

    r, c = 0.05, 2e-4

    def cost(i):
        return r * (0.3 if i < 50 else 1.0) + c * (i + 1)

    def fake_sample(w, its, threads=0):
        return sum(cost(i) for i in range(its)), {"outer_its": its}, 4

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)

    for J in (500, 781, 1270):
        exact = sum(cost(i) for i in range(J))
        est, cores, how = bench.oracle_estimate(None, 400, J)
        assert abs(est - exact) <= 1e-9 * exact, (J, est, exact)
        assert cores == 4 and f"J={J}" in how
        # the former fit on the first 100 and 200 iterations overshoots this model
        t1, t2 = fake_sample(None, 100)[0], fake_sample(None, 200)[0]
        b = 2.0 * (t2 / 200 - t1 / 100) / 100
        a = t1 / 100 - b * 50
        assert a * J + b * J * J / 2 > 1.05 * exact
    est, _, how = bench.oracle_estimate(None, 400, 300)      # sample reaches J: no extrapolation
    assert "scaled linearly" in how
