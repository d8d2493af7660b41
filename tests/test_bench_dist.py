"""The benchmark's multi-rank path (replicas, one event per rank) on CPU:
two gloo ranks agree on the slowest rank's time and on the aggregate
throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [12.0, 20.0][rank]
    ms_max, value = bench.aggregate(ms_local, 1000, 50, world)
    q.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 20.0
        assert value == pytest.approx(2 * 1000 * 50 / 0.020)


def test_single_rank_aggregate():
    import bench
    ms, v = bench.aggregate(10.0, 100, 10, 1)
    assert ms == 10.0 and v == pytest.approx(100 * 10 / 0.010)


def test_compulsory_bytes_per_site():
    """The roofline's algorithmic bytes: read and write 3 links and 3 E
    fields once per site (SU(2): 4 reals per link, SU(3): 18; fields
    nc^2 - 1 reals)."""
    import bench
    assert bench.bytes_per_site(3, 4) == 624
    assert bench.bytes_per_site(3, 8) == 1248
    assert bench.bytes_per_site(2, 8) == 336
    assert bench.bytes_per_site(2, 4) == 168


def test_profile_figures_are_tied_to_the_kernel_sources(monkeypatch):
    """The committed ncu figures (DRAM bytes, FFMA count) are used only for
    the captured workload and only while the step kernel's sources hash to
    the captured value; otherwise the bench reports them as null."""
    import bench
    e = bench.load_profile_entry("su3_512x64x64", "fp32", 512)
    if e is not None:
        assert e["dram_bytes_per_launch"] > 0 and e.get("ffma_per_launch", 1) > 0
    assert bench.load_profile_entry("su3_512x64x64", "fp32", 160) is None
    assert bench.load_profile_entry("su3_512x64x64", "fp64", 512) is None
    # and only for the kernel they were taken on
    if e is not None:
        assert bench.load_profile_entry("su3_512x64x64", "fp32", 512, e["kernel"]) is not None
        assert bench.load_profile_entry("su3_512x64x64", "fp32", 512, "k_step_plaq") is None
    monkeypatch.setattr(bench, "step_kernel_hash", lambda: "0" * 16)
    assert bench.load_profile_entry("su3_512x64x64", "fp32", 512) is None
    assert bench.load_traffic("su3_512x64x64", "fp32", 512) is None
