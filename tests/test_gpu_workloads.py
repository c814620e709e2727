"""GPU runs of the remaining measurement workloads: the water-like box and the 1e7-particle system.

Accuracy is checked against the FP64 oracle (converged Ewald sum) at sampled targets; the water
box additionally checks the autograd energy gradient by central finite differences.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from conftest import require_library  # noqa: E402

pe = require_library()
from oracle import exact  # noqa: E402
from workloads import uniform_neutral, water_box  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def water():
    x, q, L = water_box()
    tg = np.linspace(0, len(q) - 1, 48).astype(np.int64)
    ref = exact.pswf_exact(x, q, L, targets=tg)
    return x, q, L, tg, ref


def test_water_mixed_tol_1e6(water):
    """33,000 rigid 3-site molecules, 9.96 nm box, MIXED at tol 1e-6 (intramolecular pairs included)."""
    x, q, L, tg, ref = water
    plan = pe.Plan(L, len(q), 1e-6, precision="mixed")
    phi, F, E = plan.eval(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    assert _rel(phi[tg], ref[0]) <= 2e-6
    assert _rel(F[tg], ref[3]) <= 2e-6
    assert np.isfinite(E)


def test_water_autograd_forces_by_finite_differences(water):
    x, q, L, tg, ref = water
    plan = pe.Plan(L, len(q), 1e-10, precision="fp64")
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    qt = torch.tensor(q, device="cuda")
    E = pe.energy(xt, qt, plan)
    E.backward()
    g = xt.grad.cpu().numpy()
    h = 1e-4   # balances truncation (h^2 |E'''|) against rounding (eps |E| / h) for |E| ~ 1e5
    for i, d in [(0, 0), (1, 1), (50_001, 2), (98_999, 0)]:
        xp = x.copy()
        xm = x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        Ep = plan.eval(torch.tensor(xp, device="cuda"), qt)[2]
        Em = plan.eval(torch.tensor(xm, device="cuda"), qt)[2]
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - g[i, d]) <= 1e-5 * max(1.0, np.max(np.abs(g)))


def test_water_autograd_forces_float32_path(water):
    """The water box's headline form (tol 1e-6, float32 path): the autograd gradient of E (-F of the
    float32 path) against central differences of the FP64 energy (tol 1e-10, the reference gradient);
    the float32 gradient must carry no more than the path's force error (2 tol of max |F|)."""
    x, q, L, tg, ref = water
    plan = pe.Plan(L, len(q), 1e-6, precision="mixed")
    assert plan.params.precision == pe.EWALD_MIXED
    exact_plan = pe.Plan(L, len(q), 1e-10, precision="fp64")
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    qt = torch.tensor(q, device="cuda")
    E = pe.energy(xt, qt, plan)
    E.backward()
    g = xt.grad.cpu().numpy()
    gmax = np.max(np.abs(g))
    h = 1e-4
    for i, d in [(0, 0), (2, 1), (33_003, 2), (98_997, 0), (61_000, 1)]:
        xp = x.copy()
        xm = x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        Ep = exact_plan.eval(torch.tensor(xp, device="cuda"), qt)[2]
        Em = exact_plan.eval(torch.tensor(xm, device="cuda"), qt)[2]
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - g[i, d]) <= 2e-6 * gmax + 1e-5, (i, d, fd, g[i, d])


def test_large_system_1e7_tol_1e8():
    """n = 1e7 uniform neutral charges, tol 1e-8: sampled targets against the oracle, sum F = 0."""
    n = 10_000_000
    x, rho, L = uniform_neutral(n, seed=5)
    plan = pe.Plan(L, n, 1e-8, precision="mixed")
    phi, F, E = plan.eval(torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda"))
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(F)) and np.isfinite(E)
    tg = np.linspace(0, n - 1, 24).astype(np.int64)
    ref = exact.pswf_exact(x, rho, L, targets=tg)
    assert _rel(phi[tg], ref[0]) <= 2e-8
    assert _rel(F[tg], ref[3]) <= 2e-8
    assert np.max(np.abs(F.sum(axis=0))) <= 1e-6 * np.sqrt(n) * np.sqrt(np.mean(F ** 2))
