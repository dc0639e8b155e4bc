"""bench.py's multi-rank logic on CPU with two gloo ranks: the job's step time is the maximum
over ranks, the value is the whole job's throughput, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.reduce_max_ms(3.0 + 2.0 * rank)          # rank 0: 3 ms, rank 1: 5 ms
        val = bench.job_value(ms, world, 4_194_304)
        args = type("A", (), {"steps": 1, "warmup": 0})()
        ref = bench.run_reference(args, rank, world) if rank != 0 else "rank0"
        dist.barrier()
        out[rank] = (ms, val, ref is None or ref == "rank0")
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_and_value():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, val, ref_ok = out[r]
        assert ms == pytest.approx(5.0)
        assert val == pytest.approx(2 * 4_194_304 / 5e-3 / 1e6)
        assert ref_ok


def test_single_process_identity():
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_max_ms(7.25) == 7.25
    assert bench.job_value(5.0, 1, 1_000_000) == pytest.approx(200.0)


def test_cpu_baseline_fields_on_a_small_workload():
    """The oracle leg reports its thread count, per-phase times and a one-thread figure, and
    scales the samples to a whole step (a small workload, so the oracle finishes at once)."""
    import bench
    import oracle
    cfg = dict(bench.HEADLINE)
    cfg.update(H=96, W=80, D=32, k=8, th=24, tw=20, iters=3, M=6, n_sp=40)
    q, T, _, bank = bench.make_workload("cpu", cfg)
    cb = bench.cpu_baseline(q, T, cfg, bank, one_thread=True)
    assert cb["kind"] == "oracle" and cb["unit"] == "Mpix/s" and cb["value"] > 0
    assert cb["cores"] == oracle.set_threads(0) >= 1
    assert set(cb["phases_s"]) == {"fit_one_lloyd_step", "assign_640_px", "score_1024_windows"}
    assert cb["one_thread"]["value"] > 0 and set(cb["one_thread"]["phases_s"]) == set(cb["phases_s"])
    # the step estimate is the phases scaled to the workload
    ph = cb["phases_s"]
    L, HO, WO = 96 * 80, 96 - 24 + 1, 80 - 20 + 1
    est = ph["fit_one_lloyd_step"] * 3 + ph["assign_640_px"] * (L + 24 * 20) / 640 + \
        ph["score_1024_windows"] * HO * WO / 1024
    assert abs(est - cb["step_s_estimate"]) <= 0.01 + 0.01 * est


def test_launch_count_claim_matches_the_launch_sequence():
    """gpu_launches counts the library's kernels per step.  The headline launch list
    (profiles/launches_bench_headline_2048.md) shows 78 per BF16 step:
    - 12 each of prep centroids, contraction and re-scoring;
    - 3 of prep mean (the fit's first Lloyd step, the template and the query assignment);
    - 10 each of the two sort kernels and the update;
    - one each of gather, template responses, stats, row carries, band sums, band prefix,
      write pass, score and argmax."""
    import bench
    assert bench.kernels_per_step(bench.HEADLINE, "bf16") == 12 * 3 + 3 + 10 * 3 + 9


def test_reference_arm_line_on_rank_zero(monkeypatch):
    """The reference arm's JSON line on rank 0 (the oracle's bounded sample stubbed out so the
    test is quick): the base contract's keys, impl = reference, and its own e2e and
    cpu_baseline objects."""
    import json
    import bench

    def fake_workload(dev, cfg):
        return None, None, {"top_left": (0, 0)}, None

    def fake_baseline(q, T, cfg, bank, **kw):
        return {"value": 0.25, "unit": "Mpix/s", "cores": 4, "kind": "oracle", "sample": "stub",
                "step_s_estimate": 16.0, "phases_s": {}}

    monkeypatch.setattr(bench, "make_workload", fake_workload)
    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)
    args = type("A", (), {"steps": 2, "warmup": 1})()
    line = bench.run_reference(args, 0, 1)
    json.dumps(line)                                      # one JSON line
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] == 0.25 and line["steps"] == 2
    assert line["e2e"]["value"] == 0.25 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == 0.25

