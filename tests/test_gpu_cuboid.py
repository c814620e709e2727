"""Cuboid boxes (Remark on cuboid domains, Sec. 6.1): the CUDA path against the cuboid oracle.

Stage parity uses the oracle's step-by-step Alg. 2 with the plan's own per-axis grids; end-to-end
parity uses the converged cuboid Ewald sum (relative l2 of phi and F, relative E, <= 2 tol).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from conftest import require_library  # noqa: E402

pe = require_library()
from oracle import exact  # noqa: E402
from oracle.alg2 import Alg2  # noqa: E402

BOX = (1.0, 1.25, 0.75)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _system(n, seed, box=BOX):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3)) * np.array(box)
    q = rng.uniform(-1, 1, n)
    return x, q - q.mean()


def _run(x, q, box, tol, prec, **opts):
    plan = pe.Plan(box, len(q), tol, precision=prec, **opts)
    phi, F, E = plan.eval(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"))
    return plan, phi.cpu().numpy(), F.cpu().numpy(), E


@pytest.fixture(scope="module")
def stage_case():
    x, q = _system(1500, 11)
    plan, phi, F, E = _run(x, q, BOX, 1e-12, "fp64")
    p = plan.params
    A = Alg2(BOX, list(p.grid), p.P, p.cs, p.cw, p.rc)
    return plan, A, x, q, phi, F, E, A.total(x, q, stages=True)


def test_stage_spread_grid(stage_case):
    plan, A, x, q, phi, F, E, ref = stage_case
    assert len(set(plan.params.grid)) >= 2
    a_gpu = plan.debug_grid(0).reshape(ref[4]["a"].shape)
    a_ref = ref[4]["a"]
    assert np.max(np.abs(a_gpu - a_ref)) <= 50 * plan.params.fit_tol * np.max(np.abs(a_ref))


def test_stage_scaled_inverse_grid(stage_case):
    """b in the norm interpolation sees (each Fourier mode weighted by the window transform)."""
    plan, A, x, q, phi, F, E, ref = stage_case
    b_ref = ref[4]["b"]
    b_gpu = plan.debug_grid(1).reshape(b_ref.shape)
    W = A.window_ft(0)[:, None, None] * A.window_ft(1)[None, :, None] * A.window_ft(2)[None, None, :]
    d = np.fft.fftn(b_gpu - b_ref) * W
    r = np.fft.fftn(b_ref) * W
    assert np.linalg.norm(d) <= 1e-11 * np.linalg.norm(r)


def test_stage_total_vs_cpu_alg2(stage_case):
    plan, A, x, q, phi, F, E, ref = stage_case
    assert _rel(phi, ref[0]) <= 1e-10
    assert _rel(F, ref[3]) <= 1e-9
    assert abs(E - ref[2]) <= 1e-10 * abs(ref[2])


@pytest.mark.parametrize("tol,prec", [(1e-6, "mixed"), (1e-8, "fp64"), (1e-10, "mixed"), (1e-10, "fp64")])
def test_end_to_end_vs_exact(tol, prec):
    x, q = _system(3000, 2)
    ref = exact.pswf_exact(x, q, BOX)
    plan, phi, F, E = _run(x, q, BOX, tol, prec)
    assert _rel(phi, ref[0]) <= 2 * tol
    assert _rel(F, ref[3]) <= 2 * tol
    assert abs(E - ref[2]) <= 2 * tol * abs(ref[2])


def test_elongated_box_and_wrapping():
    """A 2:1:1 box (a supercell of the unit cube), positions given outside the box."""
    box = (2.0, 1.0, 1.0)
    x, q = _system(2000, 3, box)
    ref = exact.pswf_exact(x, q, box)
    shifted = x + np.array([4.0, -3.0, 7.0]) * np.array(box)
    plan, phi, F, E = _run(shifted, q, box, 1e-8, "fp64")
    assert _rel(phi, ref[0]) <= 2e-8 and _rel(F, ref[3]) <= 2e-8


def test_equal_edges_match_the_cube_api():
    x, q = _system(2000, 4, (1.1, 1.1, 1.1))
    _, phi_a, F_a, E_a = _run(x, q, 1.1, 1e-8, "fp64")
    _, phi_b, F_b, E_b = _run(x, q, (1.1, 1.1, 1.1), 1e-8, "fp64")
    assert _rel(phi_b, phi_a) <= 1e-14 and _rel(F_b, F_a) <= 1e-13
