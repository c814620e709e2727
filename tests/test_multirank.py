"""Host logic of the multi-GPU bench path (replicas, max-over-ranks timing) on gloo, world size 2, CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1.5 + rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, device="cpu")
    value = bench.aggregate_value(100_000, world, ms)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.5
    assert out[0][1] == pytest.approx(2 * 100_000 / 2.5e-3)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.aggregate_value(10, 1, 1.0) == pytest.approx(1e4)


def test_stage_roofline_report():
    """The bench's per-stage roofline report: algorithmic bytes and flops of the bench plan (host only)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    class Params:
        P, deg_w, deg_r, tile, grid = 12, 8, 11, 8, (96, 96, 96)

    n = 100_000
    stages = {"sort": 0.04, "spread": 0.07, "halo": 0.033, "scale": 0.008, "interp": 0.105, "short": 0.16,
              "energy": 0.012}
    rep = bench.stage_rooflines(stages, Params, n, 6.1e6, "f32")
    rows = {r["stage"]: r for r in rep["stages"]}
    assert set(rows) == set(stages)
    # spreading: records in, grid out; P^3 + P^2 + 3 P (d_w + 1) multiply-adds per particle
    assert rows["spread"]["bytes"] == n * 24 + 96 ** 3 * 4
    assert rows["spread"]["flops"] == n * 2 * (12 ** 3 + 12 ** 2 + 3 * 12 * 9)
    # halo: 12^3 tiles of 19^3 slab values in, the grid out
    assert rows["halo"]["bytes"] == 12 ** 3 * 19 ** 3 * 4 + 96 ** 3 * 4
    for r in rows.values():
        assert 0 < r.get("frac_hbm", 1e-9) < 1 and 0 < r.get("frac_alu", 1e-9) < 1
    # a broken input never raises: the bench line must still print
    assert "error" in bench.stage_rooflines(stages, None, n, 6.1e6, "f32")
