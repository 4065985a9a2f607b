"""The multi-rank path of bench.py on the CPU: two gloo ranks (world size 2, 127.0.0.1).

Under torchrun every rank codes its own stripes (weak scaling, no collective on the data path):
rank r's stripe bytes are its own contiguous shard of the seeded synthetic stream and its erasure
patterns come from its own seed; the step time is the maximum over ranks and the whole-job value
counts every rank's bytes over that time. These are the helpers bench.py calls; here they run in
two spawned processes joined by a gloo process group.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1709_00178_gb300.synth import BASE_SEED, synth_bytes
        stripe_bytes, stripes = 1000, 3
        off, pseed = bench.rank_shard(rank, stripe_bytes, stripes)
        shard = synth_bytes(BASE_SEED + 1, off, stripes * stripe_bytes)
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, world, dist, "cpu")
        value = bench.whole_job_gbs(world, 2e9, ms)
        pats = bench.patterns(pseed, 8, 10, 4)
        dist.barrier()
        out.put((rank, off, bytes(shard), ms, value, pats))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_time_and_aggregate():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = out.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_1709_00178_gb300.synth import BASE_SEED, synth_bytes
    # shards: contiguous, disjoint, together the stream's first world * shard bytes
    shard = 3 * 1000
    assert [res[r][1] for r in range(world)] == [r * shard for r in range(world)]
    whole = synth_bytes(BASE_SEED + 1, 0, world * shard)
    assert res[0][2] + res[1][2] == bytes(whole)
    # the step time every rank reports is the slowest rank's; the value counts both ranks
    assert res[0][3] == res[1][3] == 15.0
    assert res[0][4] == res[1][4] == pytest.approx(world * 2e9 / 15e-3 / 1e9)
    # each rank draws its own erasure patterns: 1..m erased blocks of k + m
    assert res[0][5] != res[1][5]
    for r in range(world):
        for pat in res[r][5]:
            assert 1 <= bin(pat).count("1") <= 4 and pat < (1 << 14)


def test_traffic_record_digest_tracks_the_kernel_sources(tmp_path, monkeypatch):
    # The DRAM traffic record applies only while the sources that shape the batched coding kernels
    # are the ones it was captured with: an edit to the device code changes the digest, an edit to
    # the server (host code the bench's kernels never run) does not.
    import shutil
    import sys
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_1709_00178_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_1709_00178_gb300", "csrc"), csrc)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_source_digest()
    with open(csrc / "server.cpp", "a") as f:
        f.write("\n// host-only edit\n")
    assert bench.kernel_source_digest() == d0
    with open(csrc / "ring_staged.cuh", "a") as f:
        f.write("\n// device edit\n")
    assert bench.kernel_source_digest() != d0
