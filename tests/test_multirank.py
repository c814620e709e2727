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
        P, deg_w, deg_r, tile, grid, precision = 12, 8, 11, 8, (96, 96, 96), 1

    n = 100_000
    stages = {"sort": 0.04, "spread": 0.07, "halo": 0.033, "scale": 0.008, "interp": 0.105, "short": 0.16,
              "energy": 0.012}
    rep = bench.stage_rooflines(stages, Params, n, 6.1e6, "f32")
    rows = {r["stage"]: r for r in rep["stages"]}
    assert set(rows) == set(stages)
    # spreading: records in, grid out; P^3 + P^2 + 3 P (d_w + 1) multiply-adds per particle
    assert rows["spread"]["bytes"] == n * 24 + 96 ** 3 * 4
    assert rows["spread"]["flops"] == n * 2 * (12 ** 3 + 12 ** 2 + 3 * 12 * 9)
    # halo: x-chains of K = 4 tiles: heads of 8 x 19^2 values per tile, tails of 11 x 19^2 per chain in,
    # the grid out
    assert rows["halo"]["bytes"] == (12 ** 3 * 8 * 19 ** 2 + 12 ** 3 // 4 * 11 * 19 ** 2) * 4 + 96 ** 3 * 4
    for r in rows.values():
        assert 0 < r.get("frac_hbm", 1e-9) < 1 and 0 < r.get("frac_alu", 1e-9) < 1
    # a broken input never raises: the bench line must still print
    assert "error" in bench.stage_rooflines(stages, None, n, 6.1e6, "f32")


# ------------------------------------------------ one batch of independent systems over two ranks --
def _oracle_evaluator(systems):
    """Evaluates the listed systems of a batch on the CPU with the converged oracle (a stand-in for the
    GPU evaluation: deterministic, so a split batch must reproduce the single-rank results bit for bit)."""
    from oracle import exact

    def evaluate(indices):
        out = []
        for i in indices:
            x, rho, L = systems[i]
            phi, _, E, F = exact.pswf_exact(x, rho, L, cs=20.0, rc_frac=0.45)
            out.append((phi, F, E))
        return out
    return evaluate


def _small_batch():
    from workloads import batched_systems
    return batched_systems(nsys=7, seed=3, nmin=20, nmax=90)


def _shard_worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from conftest import require_library
    require_library()
    from paper_2602_16591_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    systems = _small_batch()
    ns = [len(s[1]) for s in systems]
    costs = shard.batch_costs([s[2] for s in systems], ns, 1e-6)
    calls = []
    ev = _oracle_evaluator(systems)

    def evaluate(indices):
        calls.append(list(indices))
        return ev(indices)
    phi, F, E = shard.evaluate_sharded(evaluate, ns, costs, rank, world)
    out[rank] = (phi.tobytes(), F.tobytes(), E.tobytes(), calls)
    dist.barrier()
    dist.destroy_process_group()


def test_batch_split_over_two_ranks_reproduces_single_rank():
    """A batch split over two gloo ranks (no exchange while evaluating; results gathered on the host)
    gives every rank the single-rank phi, F and E bit for bit, each system evaluated exactly once."""
    from conftest import require_library
    require_library()
    import numpy as np
    from paper_2602_16591_gb300 import shard
    systems = _small_batch()
    ns = [len(s[1]) for s in systems]
    costs = shard.batch_costs([s[2] for s in systems], ns, 1e-6)
    ref = shard.evaluate_sharded(_oracle_evaluator(systems), ns, costs, 0, 1)
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        assert out[r][0] == ref[0].tobytes() and out[r][1] == ref[1].tobytes() and out[r][2] == ref[2].tobytes()
    done = sorted(i for r in range(world) for c in out[r][3] for i in c)
    assert done == list(range(len(systems)))            # every system once, on exactly one rank
    assert all(len(out[r][3]) == 1 and out[r][3][0] for r in range(world))


def test_shard_assignment_balances_cost():
    """Longest-processing-time packing: deterministic, complete, and within 4/3 of the optimum bound."""
    from conftest import require_library
    require_library()
    import numpy as np
    from paper_2602_16591_gb300 import shard
    from workloads import batched_systems
    systems = batched_systems(nsys=256, seed=0)
    ns = [len(s[1]) for s in systems]
    costs = shard.batch_costs([s[2] for s in systems], ns, 1e-6, precision="mixed")
    for world in (2, 4, 8):
        share = shard.assign(costs, world)
        assert share == shard.assign(costs, world)
        assert sorted(i for s in share for i in s) == list(range(256))
        loads = [sum(costs[i] for i in s) for s in share]
        bound = max(sum(costs) / world, max(costs))
        assert max(loads) <= 4.0 / 3.0 * bound
    # the model grows with n (up to the grid rounding of m, which moves the FFT term): the most
    # expensive system is within 10% of the largest n, and cost and n are rank-correlated
    assert ns[int(np.argmax(costs))] >= 0.9 * max(ns)
    rank_n, rank_c = np.argsort(np.argsort(ns)), np.argsort(np.argsort(costs))
    assert np.corrcoef(rank_n, rank_c)[0, 1] > 0.99


def _edge_worker(rank, world, port, nsys, fail_rank, out):
    import sys
    from datetime import timedelta
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from conftest import require_library
    require_library()
    from paper_2602_16591_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    # a short collective timeout: a rank left waiting would end the test with an error, not hang it
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
    systems = _small_batch()[:nsys]
    ns = [len(s[1]) for s in systems]
    costs = shard.batch_costs([s[2] for s in systems], ns, 1e-6)
    ev = _oracle_evaluator(systems)

    def evaluate(indices):
        if rank == fail_rank:
            raise ValueError("evaluation failed on purpose")
        return ev(indices)
    try:
        phi, F, E = shard.evaluate_sharded(evaluate, ns, costs, rank, world)
        out[rank] = ("ok", phi.tobytes(), F.tobytes(), E.tobytes(), len(shard.assign(costs, world)[rank]))
    except RuntimeError as e:
        out[rank] = ("error", str(e))
    dist.destroy_process_group()


def _run_edge(world, nsys, fail_rank):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_edge_worker, args=(world, port, nsys, fail_rank, out), nprocs=world,
                       start_method="spawn", join=True)
    return dict(out)


def test_failed_rank_is_reported_to_every_rank():
    """A rank whose evaluation raises joins the host gather with its error: every rank raises an error
    naming it, and none waits for the collective's timeout."""
    import time
    t0 = time.perf_counter()
    out = _run_edge(world=2, nsys=4, fail_rank=1)
    assert time.perf_counter() - t0 < 50
    for r in range(2):
        assert out[r][0] == "error"
        assert "rank 1 failed" in out[r][1] and "evaluation failed on purpose" in out[r][1]


def test_more_ranks_than_systems():
    """Three ranks, two systems: one rank has an empty share and still receives the whole batch's
    results, equal bit for bit to the single-rank evaluation."""
    from conftest import require_library
    require_library()
    from paper_2602_16591_gb300 import shard
    systems = _small_batch()[:2]
    ns = [len(s[1]) for s in systems]
    costs = shard.batch_costs([s[2] for s in systems], ns, 1e-6)
    ref = shard.evaluate_sharded(_oracle_evaluator(systems), ns, costs, 0, 1)
    out = _run_edge(world=3, nsys=2, fail_rank=-1)
    assert sorted(out[r][4] for r in range(3)) == [0, 1, 1]       # systems per rank
    for r in range(3):
        assert out[r][0] == "ok"
        assert out[r][1] == ref[0].tobytes() and out[r][2] == ref[1].tobytes() and out[r][3] == ref[2].tobytes()
