"""CPU tests of the C ABI's host side: exported symbols, the planner's PSWF, Alg. 3, fits, tables.

Everything here runs without a GPU (the library's host entry points make no CUDA call).
"""
import math
import os
import re

import numpy as np
import pytest
from scipy.special import lambertw

import paper_2602_16591_gb300 as pe
from oracle import params as oparams
from oracle.alg2 import Alg2
from oracle.pswf import PSWF
from oracle.split import PSWFSplit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(ewald_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = _declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(pe.lib, n), n


@pytest.mark.parametrize("c", [1.0, 6.0, 14.0, 22.0, 31.0])
def test_planner_pswf_matches_oracle(c):
    """App. B solver (Sturm bisection + inverse iteration) vs the oracle's dense eigensolver."""
    x = np.linspace(-1, 1, 33)
    psi, dpsi, chi, lam = pe.pswf_eval(c, x)
    f = PSWF(c)
    assert np.max(np.abs(psi - f.psi(x))) <= 1e-13 * f.psi0
    assert np.max(np.abs(dpsi - f.dpsi(x))) <= 1e-12 * np.max(np.abs(f.dpsi(x)))
    assert abs(chi - f.chi) <= 1e-12 * max(1, f.chi)
    assert abs(lam / f.lam - 1) <= 1e-13


@pytest.mark.parametrize("z", [1e-3, 0.5, 7.0, 1e6, 1e30])
def test_lambertw_principal(z):
    assert abs(pe.lambertw(0, z) - float(np.real(lambertw(z, 0)))) <= 1e-14 * max(1, abs(np.real(lambertw(z, 0))))


@pytest.mark.parametrize("z", [-0.35, -0.1, -1e-5, -1e-14, -1e-200])
def test_lambertw_lower(z):
    ref = float(np.real(lambertw(z, -1)))
    assert abs(pe.lambertw(-1, z) - ref) <= 1e-13 * abs(ref)


CFGS = [(1.0, 1000, 1e-6), (1.0, 512, 1e-6), (1.0, 100_000, 1e-4), (1.0, 100_000, 1e-6), (1.0, 100_000, 1e-10),
        (1.0, 100_000, 1e-12), (9.96, 99_000, 1e-6), (1.0, 10_000_000, 1e-8)]


@pytest.mark.parametrize("L,n,tol", CFGS)
def test_plan_params_match_oracle_alg3(L, n, tol):
    p = pe.plan_params(L, n, tol)
    q = oparams.plan(L, n, tol, tol_safety=0.25, grid_density=3.0)
    assert (p.m, p.P) == (q["m"], q["P"])
    for k in ("rc", "cs", "cw", "alpha", "h"):
        assert abs(getattr(p, k) / q[k] - 1) <= 1e-11, k
    assert p.tile == 4 and p.m % p.tile == 0
    assert p.ncell >= 1 and p.L / p.ncell >= p.rc / p.sr_reach - 1e-15


@pytest.mark.parametrize("L,n,tol", [c for c in CFGS if c[2] >= 1e-7])
def test_mixed_plan_params_match_oracle_alg3(L, n, tol):
    """float32 plans round m to a multiple of their tile edge 8."""
    p = pe.plan_params(L, n, tol, precision="mixed")
    q = oparams.plan(L, n, tol, tol_safety=0.25, grid_density=3.0, mult=8)
    assert p.precision == pe.EWALD_MIXED and p.tile == 8 and p.m % 8 == 0
    assert (p.m, p.P) == (q["m"], q["P"])
    for k in ("rc", "cs", "cw", "alpha", "h"):
        assert abs(getattr(p, k) / q[k] - 1) <= 1e-11, k


def test_plan_rejects_bad_arguments():
    for args in [(0.0, 100, 1e-6), (1.0, 1, 1e-6), (1.0, 100, 1e-1), (1.0, 100, 1e-15), (-1.0, 100, 1e-6)]:
        with pytest.raises(pe.EwaldError) as ei:
            pe.plan_params(*args)
        assert ei.value.code == pe.EWALD_EINVAL
    with pytest.raises(pe.EwaldError) as ei:
        pe.plan_params(1.0, 10 ** 12, 1e-6)        # grid beyond the library limit
    assert ei.value.code == pe.EWALD_ETOOBIG


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-6), ("fp64", 1e-6), ("fp64", 1e-10), ("fp64", 1e-12)])
def test_window_fit_error(prec, tol):
    """Piecewise Horner window (Remark in Sec. 4.3) against the exact psi of the oracle."""
    p = pe.plan_params(1.0, 100_000, tol, precision=prec)
    z = np.linspace(-1, 1, 801)
    w, dw = pe.window_fit(p, z)
    f = PSWF(p.cw)
    a = np.arange(p.P)
    s = (z[:, None] + p.P - 1 - 2 * a[None, :]) / p.P
    assert np.max(np.abs(w - f.psi(s) / f.psi0)) <= p.fit_tol
    ref_d = f.dpsi(s) / (f.psi0 * p.alpha)
    assert np.max(np.abs(dw - ref_d)) <= p.fit_tol * np.max(np.abs(ref_d)) * 1.01


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-6), ("fp64", 1e-10)])
def test_radial_fit_error(prec, tol):
    p = pe.plan_params(1.0, 100_000, tol, precision=prec)
    sp = PSWFSplit(p.cs, p.rc)
    r = np.linspace(0.02 * p.rc, 0.999 * p.rc, 500)
    R, G = pe.radial_fit(p, r)
    Rr, dRr = sp.R_and_dR(r)
    # R = 1/r - P1: absolute error of P1 is bounded by fit_tol * max|P1| ~ fit_tol * 3/rc
    # plus a few ulps of the exact 1/r, 1/r^3 terms, which dominate at small r
    assert np.max(np.abs(R - Rr) - 4e-16 * np.abs(Rr)) <= 4 * p.fit_tol / p.rc
    Gr = -dRr / r
    assert np.max(np.abs(G - Gr) - 4e-16 * np.abs(Gr)) <= 4 * p.fit_tol * 10 / p.rc ** 3


@pytest.mark.parametrize("L,n,tol", [(1.0, 1000, 1e-6), (1.0, 8000, 1e-10)])
def test_scale_table_matches_oracle(L, n, tol):
    """Alg. 2 step 3 table vs the oracle's S(k) (same (m, P, cs, cw, rc); ball |k| <= m/2)."""
    p = pe.plan_params(L, n, tol)
    S = pe.scale_table(p)
    A = Alg2(L, p.m, p.P, p.cs, p.cw, p.rc)
    So = A.scaling()[:, :, : p.m // 2 + 1]
    # the R2C half spectrum's last plane iz = m/2 is k_z = -m/2 in I_m; S is even in k_z
    So = So.copy()
    So[:, :, p.m // 2] = A.scaling()[:, :, p.m // 2]
    nz = So != 0
    assert np.all((S != 0) == nz)
    # S = (Mhat/V) / D with D = prod_i (phihat_i/h)^2.  Where Mhat or phihat are ~e^{-c} both sides
    # lose digits to cancellation, so S is compared through the Mhat it encodes: the error of
    # S * D must be tiny against max Mhat/V (that is what enters phi, Alg. 2 steps 3-5).
    k = A.kgrid()
    ph1 = A.alpha * A.win.cos_transform(2 * np.pi * k / L * A.alpha) / (A.win.psi0 * A.h)
    D = (ph1[:, None, None] * ph1[None, :, None] * ph1[None, None, :])[:, :, : p.m // 2 + 1] ** 2
    M = So * D
    assert np.max(np.abs(S * D - M)) <= 1e-12 * np.max(M)


def test_precision_paths():
    """MIXED below tol 1e-7 runs the float-float kernels; float-float plans size their fits like FP64."""
    for tol in (1e-8, 1e-10, 1e-12):
        pm = pe.plan_params(1.0, 50_000, tol, precision="mixed")
        pf = pe.plan_params(1.0, 50_000, tol, precision="floatfloat")
        p64 = pe.plan_params(1.0, 50_000, tol, precision="fp64")
        assert pm.precision == pf.precision == pe.EWALD_FLOATFLOAT
        assert p64.precision == pe.EWALD_FP64
        for k in ("m", "P", "deg_w", "deg_r", "fit_tol", "rc"):
            assert getattr(pf, k) == getattr(p64, k)
    assert pe.plan_params(1.0, 50_000, 1e-6, precision="mixed").precision == pe.EWALD_MIXED
    assert pe.plan_params(1.0, 50_000, 1e-6, precision="floatfloat").precision == pe.EWALD_FLOATFLOAT
    with pytest.raises(pe.EwaldError):
        pe.plan_params(1.0, 50_000, 1e-6, precision=7)


def test_opts_defaults_and_autotune_validation():
    import ctypes
    o = pe.make_opts()
    assert o.autotune == 0 and o.grid_density == 3.0 and o.tol_safety == 0.25 and o.window_extra == 0
    o.autotune = 2
    p = pe.ewald_params()
    assert pe.lib.ewald_plan_params(1.0, 1000, 1e-6, ctypes.byref(o), ctypes.byref(p)) == pe.EWALD_EINVAL


def test_batch_arguments_rejected_before_any_device_work():
    import ctypes
    h = ctypes.c_void_p()
    L = np.array([1.0, 2.0])
    n = np.array([100, 200], dtype=np.int64)
    o = pe.make_opts()
    args = lambda k, Lp, np_: (k, Lp, np_, 1e-6, ctypes.byref(o), ctypes.byref(h))  # noqa: E731
    Lp, Np = L.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p)
    assert pe.lib.ewald_plan_batch_create(*args(0, Lp, Np)) == pe.EWALD_EINVAL
    assert pe.lib.ewald_plan_batch_create(*args(5000, Lp, Np)) == pe.EWALD_EINVAL
    assert pe.lib.ewald_plan_batch_create(*args(2, None, Np)) == pe.EWALD_EINVAL
    bad = np.array([-1.0, 2.0])
    assert pe.lib.ewald_plan_batch_create(*args(2, bad.ctypes.data_as(ctypes.c_void_p), Np)) == pe.EWALD_EINVAL
    assert b"system 0" in pe.lib.ewald_last_error()
    off = np.array([0, 100, 300], dtype=np.int64)
    assert pe.lib.ewald_eval_batch(None, off.ctypes.data_as(ctypes.c_void_p), None, None, None, None, None,
                                   None) == pe.EWALD_EINVAL


# ------------------------------------------------------------------ cuboid boxes (Remark, Sec. 6.1) --
@pytest.mark.parametrize("box,n,tol,prec,mult", [((1.0, 1.25, 0.75), 5000, 1e-6, "fp64", 4),
                                                 ((1.0, 1.25, 0.75), 5000, 1e-6, "mixed", 8),
                                                 ((2.0, 1.0, 1.0), 100_000, 1e-10, "fp64", 4),
                                                 ((0.9, 1.7, 1.2), 40_000, 1e-8, "floatfloat", 4)])
def test_cuboid_plan_params_match_oracle(box, n, tol, prec, mult):
    p = pe.plan_params(box, n, tol, precision=prec)
    q = oparams.plan_box(box, n, tol, tol_safety=0.25, grid_density=3.0, mult=mult)
    assert list(p.grid) == q["m"] and p.P == q["P"] and p.deg_g > 0
    assert list(p.box) == list(box)
    for k in ("rc", "cs", "cw"):
        assert abs(getattr(p, k) / q[k] - 1) <= 1e-11, k
    for d in range(3):   # cells of edge >= rc / reach on every axis
        assert box[d] / p.cells[d] >= p.rc / p.sr_reach - 1e-15


def test_box_api_with_equal_edges_is_the_cube():
    for prec in ("fp64", "mixed"):
        a = pe.plan_params(1.3, 20_000, 1e-7, precision=prec).as_dict()
        b = pe.plan_params((1.3, 1.3, 1.3), 20_000, 1e-7, precision=prec).as_dict()
        assert a == b and a["deg_g"] == 0


def test_eval_host_output_arrays_are_checked():
    """Caller-owned outputs of Plan.eval_host: float64, C-contiguous, writeable, exact shape (host only)."""
    a = np.empty((7, 3))
    assert pe._out(a, (7, 3)) is a
    assert pe._out(None, (7,)).shape == (7,)
    for bad in (np.empty((7, 3), dtype=np.float32), np.empty((3, 7)).T, np.empty(7), [0.0] * 21):
        with pytest.raises(ValueError):
            pe._out(bad, (7, 3))
    ro = np.empty((7, 3))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        pe._out(ro, (7, 3))
