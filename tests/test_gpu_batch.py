"""Batches of independent systems (ewald_plan_batch_create / ewald_eval_batch): every system's
result equals its own single-system plan's, meets the accuracy bar against the oracle, and the
captured graph is replayed and re-captured correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from conftest import require_library  # noqa: E402

pe = require_library()
from oracle import exact  # noqa: E402
from workloads import batched_systems  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _escale(rho, phi):
    """Scale of E = rho.phi/2 for comparisons: |dE| <= |rho| |dphi| / 2 (E itself may nearly cancel)."""
    return 0.5 * float(np.linalg.norm(rho) * np.linalg.norm(phi))


def _concat(systems):
    x = np.concatenate([s[0] for s in systems])
    rho = np.concatenate([s[1] for s in systems])
    return x, rho, np.array([s[2] for s in systems]), np.array([len(s[1]) for s in systems], dtype=np.int64)


@pytest.fixture(scope="module")
def small_batch():
    return batched_systems(nsys=12, seed=3, nmin=300, nmax=4000)


@pytest.mark.parametrize("tol,prec,bar", [(1e-6, "mixed", 1e-6), (1e-10, "fp64", 1e-12), (1e-10, "mixed", 1e-11)])
def test_batch_matches_single_plans(small_batch, tol, prec, bar):
    x, rho, Ls, ns = _concat(small_batch)
    bp = pe.BatchPlan(Ls, ns, tol, precision=prec)
    phi, F, E = bp.eval(torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda"))
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    o = bp.offsets
    for b, (xb, rb, Lb) in enumerate(small_batch):
        plan = pe.Plan(Lb, len(rb), tol, precision=prec)
        p1, F1, E1 = plan.eval(torch.tensor(xb, device="cuda"), torch.tensor(rb, device="cuda"))
        assert _rel(phi[o[b]:o[b + 1]], p1.cpu().numpy()) <= bar
        assert _rel(F[o[b]:o[b + 1]], F1.cpu().numpy()) <= 10 * bar
        assert abs(E[b] - E1) <= bar * _escale(rb, phi[o[b]:o[b + 1]])


def test_batch_vs_oracle(small_batch):
    tol = 1e-6
    sys3 = [small_batch[i] for i in (0, 5, 11)]
    x, rho, Ls, ns = _concat(sys3)
    bp = pe.BatchPlan(Ls, ns, tol, precision="mixed")
    phi, F, E = bp.eval(torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda"))
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    o = bp.offsets
    for b, (xb, rb, Lb) in enumerate(sys3):
        tg = np.linspace(0, len(rb) - 1, 24).astype(np.int64)
        ref = exact.pswf_exact(xb, rb, Lb, targets=tg)
        assert _rel(phi[o[b]:o[b + 1]][tg], ref[0]) <= 2 * tol
        assert _rel(F[o[b]:o[b + 1]][tg], ref[3]) <= 2 * tol


def test_graph_replay_and_recapture(small_batch):
    x, rho, Ls, ns = _concat(small_batch)
    bp = pe.BatchPlan(Ls, ns, 1e-6, precision="mixed")
    xt, rt = torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda")
    phi0, F0, E0 = bp.eval(xt, rt)
    phi0, F0 = phi0.clone(), F0.clone()
    phi1, F1, E1 = bp.eval(xt, rt)                     # new output buffers: re-captured
    out_phi, out_F = torch.empty_like(phi1), torch.empty_like(F1)
    phi2, F2, E2 = bp.eval(xt, rt, out_phi, out_F)     # re-captured with caller buffers
    phi3, F3, E3 = bp.eval(xt, rt, out_phi, out_F)     # replayed
    o = bp.offsets
    p0 = phi0.cpu().numpy()
    esc = np.array([_escale(rho[o[b]:o[b + 1]], p0[o[b]:o[b + 1]]) for b in range(len(ns))])
    for ph, ff, ee in ((phi1, F1, E1), (phi2, F2, E2), (phi3, F3, E3)):
        assert _rel(ph.cpu().numpy(), p0) <= 1e-6
        assert _rel(ff.cpu().numpy(), F0.cpu().numpy()) <= 1e-5
        assert np.all(np.abs(ee - E0) <= 1e-6 * esc)
    # moved positions through the same buffers are picked up by the replayed graph
    x2 = x.copy()
    x2[: ns[0]] += 0.25 * Ls[0]
    xt.copy_(torch.tensor(x2, device="cuda"))
    phi4, _, E4 = bp.eval(xt, rt, out_phi, out_F)
    assert abs(E4[0] - E0[0]) <= 1e-5 * esc[0]               # translation invariance
    assert np.all(np.abs(E4[1:] - E3[1:]) <= 1e-6 * esc[1:])


def test_batch_reports_the_failing_system(small_batch):
    x, rho, Ls, ns = _concat(small_batch)
    bp = pe.BatchPlan(Ls, ns, 1e-6, precision="mixed")
    rho = rho.copy()
    k = 4
    rho[bp.offsets[k]] += 0.5
    with pytest.raises(pe.EwaldError) as ei:
        bp.eval(torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda"))
    assert ei.value.code == pe.EWALD_ENONNEUTRAL and "system %d" % k in str(ei.value)
    import ctypes
    bad = bp.offsets.copy()
    bad[1] += 1
    xt, rt = torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda")
    code = pe.lib.ewald_eval_batch(bp._h, bad.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(xt.data_ptr()),
                                   ctypes.c_void_p(rt.data_ptr()), None, None, None, None)
    assert code == pe.EWALD_EINVAL


def test_full_batch_workload():
    """256 systems, n log-uniform in [500, 20000], L = (n/100)^(1/3), tol 1e-6 (the batched workload)."""
    systems = batched_systems(nsys=256, seed=0)
    x, rho, Ls, ns = _concat(systems)
    bp = pe.BatchPlan(Ls, ns, 1e-6, precision="mixed")
    phi, F, E = bp.eval(torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda"))
    assert np.all(np.isfinite(E)) and torch.isfinite(phi).all() and torch.isfinite(F).all()
    phi = phi.cpu().numpy()
    F = F.cpu().numpy()
    for b in (0, 137):
        xb, rb, Lb = systems[b]
        tg = np.linspace(0, len(rb) - 1, 16).astype(np.int64)
        ref = exact.pswf_exact(xb, rb, Lb, targets=tg)
        o = bp.offsets
        assert _rel(phi[o[b]:o[b + 1]][tg], ref[0]) <= 2e-6
        assert _rel(F[o[b]:o[b + 1]][tg], ref[3]) <= 2e-6


def test_sharded_shares_equal_the_whole_batch_bitwise():
    """The two shares of a batch split for two GPUs (ShardedBatchPlan, evaluated one after the other on
    this GPU) give exactly the results of the whole batch in one BatchPlan: systems share nothing and
    every evaluation is deterministic, so the split is invisible in the bits."""
    from paper_2602_16591_gb300 import shard
    systems = batched_systems(nsys=12, seed=4, nmin=500, nmax=3000)
    Ls = np.array([s[2] for s in systems])
    ns = np.array([len(s[1]) for s in systems], dtype=np.int64)
    x = torch.tensor(np.concatenate([s[0] for s in systems]), device="cuda")
    rho = torch.tensor(np.concatenate([s[1] for s in systems]), device="cuda")
    phi, F, E = pe.BatchPlan(Ls, ns, 1e-6, precision="mixed").eval(x, rho)
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    results = {}
    for r in range(2):
        sp = shard.ShardedBatchPlan(Ls, ns, 1e-6, rank=r, world=2, precision="mixed")
        assert sp.share[r]
        for i, res in zip(sp.share[r], sp.eval_local(x, rho)):
            results[i] = res
    assert sorted(results) == list(range(len(systems)))
    off = np.concatenate([[0], np.cumsum(ns)])
    for i in range(len(systems)):
        assert np.array_equal(results[i][0], phi[off[i]:off[i + 1]])
        assert np.array_equal(results[i][1], F[off[i]:off[i + 1]])
        assert results[i][2] == E[i]
