"""ewald_spread_static: spreading into a caller-owned grid with no device allocation.

It serves callers that cannot call cudaMalloc when they need the grid (an external
allocator owns the GPU, or the loop cannot afford allocation-induced synchronisation).
Its output must equal the spread grid of the regular pipeline (ewald_eval, stage 0 of
ewald_debug_grid) for the same plan parameters, call after call: the entry point reuses
one static device array whose counters it has to clear itself.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from conftest import require_library  # noqa: E402

pe = require_library()
from workloads import uniform_neutral  # noqa: E402


def _spread_static(params, xt, rt):
    m = params.m
    out = torch.full((m ** 3,), float("nan"), dtype=torch.float64, device="cuda")   # caller-owned output
    stream = torch.cuda.current_stream().cuda_stream
    code = pe.lib.ewald_spread_static(ctypes.byref(params), ctypes.c_void_p(xt.data_ptr()),
                                      ctypes.c_void_p(rt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream))
    assert code == pe.EWALD_OK, pe.lib.ewald_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(m, m, m)


def test_static_spread_matches_pipeline_on_consecutive_calls():
    # consecutive calls on different systems, the second one smaller (fewer particles, fewer tiles), the
    # third back at the first's parameters: leftovers of an earlier call in the shared array (counters,
    # slabs, the cached window table) would show.  Same kernels and the same stable order as the
    # pipeline, so the grids agree bit for bit.
    cases = [(21, 5200, 1e-8), (22, 900, 1e-6), (21, 5200, 1e-8)]
    for seed, n, tol in cases:
        x, rho, L = uniform_neutral(n, seed=seed)
        xt = torch.tensor(x, device="cuda")
        rt = torch.tensor(rho, device="cuda")
        plan = pe.Plan(L, n, tol, precision="fp64")
        plan.eval(xt, rt)
        ref = plan.debug_grid(0)
        got = _spread_static(plan.params, xt, rt)
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref), np.max(np.abs(got - ref))


def test_static_spread_rejects_float32_plan_parameters():
    p = pe.plan_params(1.0, 1000, 1e-6, precision="mixed")
    assert p.tile == 8
    dummy = ctypes.c_void_p(16)                    # never dereferenced: the parameter check comes first
    code = pe.lib.ewald_spread_static(ctypes.byref(p), dummy, dummy, dummy, None)
    assert code == pe.EWALD_EINVAL
    assert b"tile 8" in pe.lib.ewald_last_error()


def test_static_spread_rejects_problems_beyond_its_scratch():
    p = pe.plan_params(1.0, 10_000_000, 1e-8)     # m = 216: the tile slabs alone exceed the array
    dummy = ctypes.c_void_p(16)                    # never dereferenced: the size check comes first
    code = pe.lib.ewald_spread_static(ctypes.byref(p), dummy, dummy, dummy, None)
    assert code == pe.EWALD_ETOOBIG
    assert b"static array" in pe.lib.ewald_last_error()


def test_static_spread_repeat_call_skips_the_table_copy():
    """A second call with the same (c_w, P, deg_w) leaves the cached window table alone: it issues no
    host-to-device copy, so it can be recorded into a CUDA graph (a copy from pageable host memory could
    not be), and the replayed graph reproduces the grid of the direct call bit for bit."""
    x, rho, L = uniform_neutral(3000, seed=5)
    xt = torch.tensor(x, device="cuda")
    rt = torch.tensor(rho, device="cuda")
    params = pe.plan_params(L, len(x), 1e-8, precision="fp64")
    ref = _spread_static(params, xt, rt)           # first call: fits and copies the table
    m = params.m
    out = torch.full((m ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
            code = pe.lib.ewald_spread_static(ctypes.byref(params), ctypes.c_void_p(xt.data_ptr()),
                                              ctypes.c_void_p(rt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(side.cuda_stream))
    assert code == pe.EWALD_OK, pe.lib.ewald_last_error().decode()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().reshape(m, m, m), ref)
