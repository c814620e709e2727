"""Splitting one batch of independent periodic systems over several GPUs (one process per GPU).

The systems of a batch share nothing (each has its own box, grid and cell list), so a batch shards
without any exchange on the data path: every rank evaluates the systems assigned to it on its own
GPU, and the per-system results (phi, F, E) are gathered on the host afterwards.  The assignment is
a deterministic longest-processing-time bin packing by the estimated cost of a system,

    cost = 6 P^3 n  (spread + interpolation)  +  100 N_nb n  (real-space pairs)  +  5 m^3 log2(m^3)  (FFTs),

with N_nb = (4/3) pi r_c^3 n / V the mean number of neighbours inside the cutoff, taken from the
host planner (Alg. 3 with the library's rules; no GPU needed).  Every rank computes the same
assignment from the same inputs, so no rank has to be told its share.
"""
import math

import numpy as np


def system_cost(params, n):
    """Estimated work of one evaluation of an n-particle system with plan parameters `params`."""
    box = [float(v) for v in params.box]
    grid = [int(v) for v in params.grid]
    V = box[0] * box[1] * box[2]
    m3 = grid[0] * grid[1] * grid[2]
    nnb = 4.0 / 3.0 * math.pi * params.rc ** 3 * n / V
    return 6.0 * params.P ** 3 * n + 100.0 * nnb * n + 5.0 * m3 * math.log2(max(m3, 2))


def assign(costs, world):
    """Longest-processing-time bin packing: systems by decreasing cost (ties: lower index first), each to
    the rank with the least load so far (ties: lower rank).  Returns one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    share = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        share[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in share]


def batch_costs(Ls, ns, tol, **opts):
    """Cost of every system of a batch from the host planner (ewald_plan_params)."""
    from . import plan_params
    return [system_cost(plan_params(float(L), int(n), tol, **opts), int(n)) for L, n in zip(Ls, ns)]


def evaluate_sharded(evaluate, ns, costs, rank, world, group=None):
    """Evaluate the systems of one batch split over `world` ranks and gather the results on every rank.

    evaluate(indices) evaluates the listed systems on this rank and returns, for each of them in order,
    a tuple (phi (n_i,), F (n_i, 3), E) of host arrays.  The gather runs over torch.distributed on the
    host (`group`: a gloo process group, or the default group); with world == 1 no process group is
    needed.  Returns phi (N,), F (N, 3) concatenated in the batch's order and E (nsys,).

    A rank whose evaluate() raises still takes part in the gather, carrying its error instead of
    results, so every rank raises RuntimeError naming the failed rank (none is left waiting for the
    collective's timeout); with world == 1 the exception propagates unchanged.
    """
    share = assign(costs, world)
    mine = share[rank]
    if world > 1:
        import torch.distributed as dist
        try:
            local, err = ({i: r for i, r in zip(mine, evaluate(mine))} if mine else {}), None
        except Exception as e:   # reported through the gather below
            local, err = {}, "%s: %s" % (type(e).__name__, e)
        gathered = [None] * world
        dist.all_gather_object(gathered, (local, err), group=group)
    else:
        gathered = [({i: r for i, r in zip(mine, evaluate(mine))} if mine else {}, None)]
    failed = [(r, e) for r, (_, e) in enumerate(gathered) if e is not None]
    if failed:
        raise RuntimeError("sharded batch: rank %d failed: %s" % failed[0])
    results = {}
    for part, _ in gathered:
        results.update(part)
    if sorted(results) != list(range(len(ns))):
        raise RuntimeError("sharded batch: systems missing after the gather")
    phi = np.concatenate([np.asarray(results[i][0], dtype=np.float64) for i in range(len(ns))])
    F = np.concatenate([np.asarray(results[i][1], dtype=np.float64).reshape(-1, 3) for i in range(len(ns))])
    E = np.array([float(results[i][2]) for i in range(len(ns))])
    return phi, F, E


class ShardedBatchPlan:
    """A batch split over the ranks of a process group: this rank plans (BatchPlan) and evaluates only
    its own systems on its current CUDA device; `eval` gathers every system's phi, F, E on the host."""

    def __init__(self, Ls, ns, tol, rank, world, group=None, precision="fp64", **opts):
        from . import BatchPlan
        self.Ls = np.ascontiguousarray(Ls, dtype=np.float64)
        self.ns = np.ascontiguousarray(ns, dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        self.rank, self.world, self.group = int(rank), int(world), group
        self.costs = batch_costs(self.Ls, self.ns, tol, precision=precision, **opts)
        self.share = assign(self.costs, self.world)
        mine = self.share[self.rank]
        self.plan = BatchPlan(self.Ls[mine], self.ns[mine], tol, precision=precision, **opts) if mine else None

    def rows(self, indices):
        """Row indices (into the batch's concatenated arrays) of the listed systems, in order."""
        return np.concatenate([np.arange(self.offsets[i], self.offsets[i + 1]) for i in indices]) \
            if len(indices) else np.zeros(0, dtype=np.int64)

    def eval_local(self, x, rho):
        """This rank's systems: x (N, 3) and rho (N,) of the WHOLE batch (device or host); returns the
        local results as a list of (phi, F, E) host arrays, one per system of this rank's share."""
        import torch
        mine = self.share[self.rank]
        if not mine:
            return []
        rows = torch.as_tensor(self.rows(mine))
        xs = torch.as_tensor(x)[rows.to(torch.as_tensor(x).device)]
        rs = torch.as_tensor(rho)[rows.to(torch.as_tensor(rho).device)]
        phi, F, E = self.plan.eval(xs, rs)
        phi, F = phi.cpu().numpy(), F.cpu().numpy()
        out, o = [], 0
        for k, i in enumerate(mine):
            m = int(self.ns[i])
            out.append((phi[o:o + m], F[o:o + m], float(E[k])))
            o += m
        return out

    def eval(self, x, rho):
        """phi (N,), F (N, 3), E (nsys,) of the whole batch on every rank (host arrays)."""
        return evaluate_sharded(lambda idx: self.eval_local(x, rho), self.ns, self.costs, self.rank, self.world,
                                self.group)
