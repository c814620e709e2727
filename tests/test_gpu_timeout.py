"""The bounded device wait: it runs out with EWALD_ETIMEOUT on a barrier that nothing arrives at, and the
CUDA context stays usable for the next evaluation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from conftest import require_library  # noqa: E402

pe = require_library()
from workloads import uniform_neutral  # noqa: E402


def test_bounded_wait_reports_timeout_and_context_survives():
    assert pe._lib.ewald_debug_wait_timeout() == pe.EWALD_ETIMEOUT
    assert b"ran out" in pe._lib.ewald_last_error()
    x, rho, L = uniform_neutral(2000, seed=1)
    plan = pe.Plan(L, len(x), 1e-4, precision="mixed", spread_kernel=2)
    phi, F, E = plan.eval(torch.tensor(x, device="cuda"), torch.tensor(rho, device="cuda"))
    assert np.all(np.isfinite(phi.cpu().numpy())) and np.isfinite(E)
