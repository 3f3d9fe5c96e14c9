"""The benchmark's multi-GPU path is replicas only: every rank decodes its own
batch, and the job's figures come from one host-side reduction. These tests
run that reduction on CPU with world_size-2 gloo ranks (every rank receives
the slowest rank's time; the job value counts all ranks' pixels), and check
that the reference arm does its work and prints its line on rank 0 only.
"""
import argparse
import json
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r: a timed total of 100 + 50 r ms, an e2e leg of 2 + r s over 3 steps
        got = bench.max_over_ranks([100.0 + 50.0 * rank, 2.0 + rank, 3.0], world)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = dict(q.get(timeout=180) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for r in range(world):
        assert res[r] == [150.0, 3.0, 3.0], (r, res[r])


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks([1.5, 7.0], 1) == [1.5, 7.0]


def test_job_value_counts_every_rank():
    # two replicas of 1e6 pixels each, the slower one took 0.5 s: 4 MPix/s
    assert bench.job_mpix_per_s(2, 1e6, 0.5) == pytest.approx(4.0)
    assert bench.job_mpix_per_s(1, 3e6, 1.0) == pytest.approx(3.0)


def test_reference_arm_on_rank0_only(monkeypatch, capsys):
    calls = []

    def fake_sample(crop):
        calls.append(crop)
        return crop * crop, 0.25

    monkeypatch.setattr(bench, "cpu_oracle_decode_sample", fake_sample)
    args = argparse.Namespace(steps=2, warmup=1, gpus=2)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(args)
    assert calls == [] and capsys.readouterr().out == ""

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("LOCAL_RANK", "0")
    bench.run_reference(args)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1 and len(calls) == 3
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is True
    assert d["value"] == pytest.approx(calls[0] ** 2 / 0.25 / 1e6)
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
