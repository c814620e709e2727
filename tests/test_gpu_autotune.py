"""Autotuning at plan creation (ewald_opts.autotune): grid density, then the real-space cell reach.
The tuned plan is one of the candidate plans, meets the accuracy bar and is not slower than the
default plan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from conftest import require_library  # noqa: E402

pe = require_library()
from oracle import exact  # noqa: E402
from workloads import uniform_neutral  # noqa: E402

CANDIDATES = (1.5, 2.0, 3.0, 4.0, 6.0, 8.0, 12.0)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _time(plan, xt, rt, reps=5):
    phi = torch.empty(len(rt), dtype=torch.float64, device="cuda")
    F = torch.empty(len(rt), 3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        plan.eval(xt, rt, phi, F, energy=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        plan.eval(xt, rt, phi, F, energy=False)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


@pytest.mark.parametrize("tol,prec", [(1e-6, "mixed"), (1e-10, "mixed")])
def test_autotuned_plan(tol, prec):
    n = 100_000
    x, rho, L = uniform_neutral(n, seed=0)
    tg = np.linspace(0, n - 1, 32).astype(np.int64)
    ref = exact.pswf_exact(x, rho, L, targets=tg)
    xt, rt = torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda")
    tuned = pe.Plan(L, n, tol, precision=prec, autotune=True)
    default = pe.Plan(L, n, tol, precision=prec)
    ms = {pe.plan_params(L, n, tol, precision=prec, grid_density=g).m for g in CANDIDATES}
    assert tuned.params.m in ms and 1 <= tuned.params.sr_reach <= 4
    phi, F, E = tuned.eval(xt, rt)
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    assert _rel(phi[tg], ref[0]) <= 2 * tol
    assert _rel(F[tg], ref[3]) <= 2 * tol
    assert _time(tuned, xt, rt) <= 1.25 * _time(default, xt, rt)
