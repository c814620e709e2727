"""CPU tests of the C ABI's host side: exported symbols, the planner's PSWF, Alg. 3, fits, tables.

Everything here runs without a GPU (the library's host entry points make no CUDA call; plan creation
is called only to check how it reports a host without a CUDA device).
"""
import math
import os
import re

import numpy as np
import pytest
from scipy.special import lambertw

from conftest import require_library
from oracle import params as oparams
from oracle.alg2 import Alg2
from oracle.pswf import PSWF
from oracle.split import PSWFSplit

pe = require_library()

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


def test_lambertw_outside_its_domain():
    """Another branch, a NaN argument or z outside a branch's domain: NaN and a message, never a
    number from an undefined logarithm."""
    for branch, z, msg in [(3, 1.0, b"branch"), (0, -1.0, b"-1/e"), (-1, 0.5, b"[-1/e, 0)"),
                           (0, float("nan"), b"not a number")]:
        assert math.isnan(pe.lambertw(branch, z))
        assert msg in pe.lib.ewald_last_error()


CFGS = [(1.0, 1000, 1e-6), (1.0, 512, 1e-6), (1.0, 100_000, 1e-4), (1.0, 100_000, 1e-6), (1.0, 100_000, 1e-10),
        (1.0, 100_000, 1e-12), (9.96, 99_000, 1e-6), (1.0, 10_000_000, 1e-8)]

# The planner runs the paper's Alg. 3 (oracle.params) with these additions of its own, each a stated
# difference from the procedure as printed (the paper leaves r_c to tuning and has no force model):
GRID_DENSITY = {8: 6.0, 4: 3.0}   # (a) r_c: fixed point r = min(c_s(r) L/(pi (g n)^(1/3)), L/2) for g = m^3/n:
#                                   6 for float32 plans (tile 8), 3 for the others (tile 4)
TOL_SAFETY = 0.25       # (b) the split and window targets are tol * 0.25
FORCE_M0 = 10.0         # (c) the split target is further multiplied by min(1, 10/m0), m0 the unrounded m
#                         (d) m is rounded up to a multiple of the spreading tile (8 for float32 plans,
#                             4 otherwise) with no prime factor above 7, and r_c re-derived from eq. csrc
#                         (e) the window (c_w, hence P) is balanced against the target of (b), not (c)


def good_size(m, mult):
    m = max(int(m), mult)
    while True:
        r = m
        for q in (2, 3, 5, 7):
            while r % q == 0:
                r //= q
        if m % mult == 0 and r == 1:
            return m
        m += 1


def library_rule(L, n, tol, mult):
    """Alg. 3 steps (oracle) with the planner's additions (a)-(e) above."""
    t = tol * TOL_SAFETY

    def cutoff(t):
        r, mstar = 0.1, (GRID_DENSITY[mult] * n) ** (1.0 / 3.0)
        for _ in range(12):
            r = min(oparams.cs_of(r, t) / (math.pi * mstar), 0.5)
        return r

    t_pot = t
    rcl = cutoff(t)
    m0 = oparams.cs_of(rcl, t) / (math.pi * rcl)
    if m0 > FORCE_M0:
        t *= FORCE_M0 / m0
        rcl = cutoff(t)
    q = oparams.alg3(1.0, t, rcl)                             # steps 1, 4 at the split target
    m = good_size(q["m"], mult)
    eff = oparams.instantiate(L, m, 0, q["cs"])               # r_c from eq. csrc after rounding
    cw = oparams.cw_of(oparams.cs_of(eff["rc"] / L, t_pot), eff["rc"] / L)     # step 2 at the target of (b)
    P = int(math.ceil(2.0 * (eff["rc"] * cw / q["cs"]) * m / L))              # steps 3, 5
    return oparams.instantiate(L, m, P, q["cs"]) | {"cw_target": cw, "t_split": t}


@pytest.mark.parametrize("L,n,tol", CFGS)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plan_params_are_alg3_plus_stated_additions(L, n, tol, prec):
    p = pe.plan_params(L, n, tol, precision=prec)
    mult = 8 if p.precision == pe.EWALD_MIXED else 4
    q = library_rule(L, n, tol, mult)
    assert p.tile == mult and p.m % p.tile == 0
    assert (p.m, p.P) == (q["m"], q["P"])
    for k in ("rc", "cs", "cw", "alpha", "h", "cw_target"):
        assert abs(getattr(p, k) / q[k] - 1) <= 1e-11, k
    assert p.ncell >= 1 and p.L / p.ncell >= p.rc / p.sr_reach - 1e-15
    assert p.L / p.cells[2] >= p.rc / p.sr_reach_z - 1e-15
    assert p.sr_reach_z == (4 if p.precision == pe.EWALD_MIXED else p.sr_reach)


@pytest.mark.parametrize("L,n,tol", CFGS)
def test_plan_differs_from_alg3_only_as_stated(L, n, tol):
    """Alg. 3 as printed at the planner's split target and unrounded cutoff gives an m that the planner
    only rounds up by (d); after rounding eq. csrc, eq. bandwidth and eq. cwP hold exactly, and P is
    eq. P_dimless for the window of (e)."""
    p = pe.plan_params(L, n, tol)
    q = library_rule(L, n, tol, 4)
    m_alg3 = math.ceil(p.cs * L / (math.pi * p.rc) - 1e-9)     # = p.m: r_c was re-derived from it
    assert m_alg3 == p.m and p.m == good_size(p.m, 4)
    assert abs(p.cs / p.rc - math.pi * p.m / L) <= 1e-12 * p.cs / p.rc
    assert abs(p.cs / p.rc - p.cw / p.alpha) <= 1e-12 * p.cs / p.rc
    assert abs(p.cw - math.pi * p.P / 2) <= 1e-12 * p.cw
    assert p.P == math.ceil(2 * p.cw_target / math.pi - 1e-12)
    # the window target (e) is looser than the split target (c): never a wider window than Alg. 3 would
    # choose for the split target itself
    assert p.cw_target <= oparams.cw_of(p.cs, p.rc / L) + 1e-9 and q["t_split"] <= tol * TOL_SAFETY


def test_plan_rejects_bad_arguments():
    for args in [(0.0, 100, 1e-6), (1.0, 1, 1e-6), (1.0, 100, 1e-1), (1.0, 100, 1e-15), (-1.0, 100, 1e-6)]:
        with pytest.raises(pe.EwaldError) as ei:
            pe.plan_params(*args)
        assert ei.value.code == pe.EWALD_EINVAL
    with pytest.raises(pe.EwaldError) as ei:
        pe.plan_params(1.0, 10 ** 12, 1e-6)        # grid beyond the library limit
    assert ei.value.code == pe.EWALD_ETOOBIG


def test_error_strings_and_thread_local_last_error():
    """Every status code has its own message (unknown codes too), and ewald_last_error() is per
    thread: a failure on another thread leaves this thread's message as it was."""
    import threading
    msgs = [pe.lib.ewald_error_string(c) for c in range(9)]
    assert all(msgs) and len(set(msgs)) == 9
    assert pe.lib.ewald_error_string(pe.EWALD_ETIMEOUT) != pe.lib.ewald_error_string(pe.EWALD_ECUDA)
    assert pe.lib.ewald_error_string(999) and pe.lib.ewald_error_string(-1)
    with pytest.raises(pe.EwaldError):
        pe.plan_params(-1.0, 100, 1e-6)
    mine = pe.lib.ewald_last_error()
    theirs = {}

    def other():
        try:
            pe.plan_params(1.0, 100, 1e-1)
        except pe.EwaldError:
            pass
        theirs["msg"] = pe.lib.ewald_last_error()

    th = threading.Thread(target=other)
    th.start()
    th.join()
    assert theirs["msg"] and theirs["msg"] != mine
    assert pe.lib.ewald_last_error() == mine


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
    """Alg. 2 step 3 table vs the oracle's S(k) (same (m, P, cs, cw, rc); modes inside the band |k| < m/2)."""
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


@pytest.mark.parametrize("box,tol", [((1.0, 1.25, 0.75), 1e-6), ((2.0, 1.0, 1.0), 1e-10)])
def test_scale_table_matches_oracle_cuboid(box, tol):
    """Cuboid boxes: the scaling table (per-axis window transforms, M-hat from the plan's gammahat
    polynomial) against the oracle's S(k) of Alg. 2 in that box, with the plan's per-axis grids: the
    same retained modes, and S times the window denominator equal to the oracle's M-hat / V within
    the polynomial fit tolerance."""
    p = pe.plan_params(box, 20_000, tol)
    assert p.deg_g > 0
    mx, my, mz = (int(v) for v in p.grid)
    S = pe.scale_table(p)
    A = Alg2(tuple(p.box), tuple(p.grid), p.P, p.cs, p.cw, p.rc)
    So = A.scaling()[:, :, : mz // 2 + 1]
    ks = [A.kgrid(d) for d in range(3)]
    KX, KY, KZ = np.meshgrid(ks[0], ks[1], np.arange(mz // 2 + 1), indexing="ij")
    t = ((KX / p.box[0]) ** 2 + (KY / p.box[1]) ** 2 + (KZ / p.box[2]) ** 2) * (2 * np.pi * p.rc / p.cs) ** 2
    clear = np.abs(t - 1.0) > 1e-9                      # modes not on the band edge itself
    assert np.all(((S != 0) == (So != 0))[clear])
    ph = [A.window_ft(d) for d in range(3)]
    D = ((ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]) ** 2)[:, :, : mz // 2 + 1]
    M = So * D
    both = (S != 0) & (So != 0)
    assert np.max(np.abs((S * D - M)[both])) <= 2 * p.fit_tol * np.max(M)


def test_host_tables_reject_parameters_the_planner_never_makes():
    """ewald_window_fit, ewald_radial_fit and ewald_scale_table take an ewald_params from the caller:
    a window support or degree out of range (a negative window degree used to crash the host), a
    non-positive or NaN bandlimit or cutoff, or a scalar m that is not grid[0] return EWALD_EINVAL."""
    import ctypes
    base = pe.plan_params(1.0, 1000, 1e-6)
    z = np.linspace(-1, 1, 5)
    r = np.linspace(0.01, 0.1, 5)
    W, DW, R, G = np.empty(5 * 24), np.empty(5 * 24), np.empty(5), np.empty(5)
    S = np.empty(base.grid[0] * base.grid[1] * (base.grid[2] // 2 + 1))
    for field, value in [("P", 0), ("P", 25), ("deg_w", -1), ("deg_w", 500), ("deg_r", -2), ("deg_g", -1),
                         ("cw", float("nan")), ("cs", -1.0), ("rc", 0.0), ("m", 0), ("alpha", 0.0)]:
        p = pe.ewald_params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(base), ctypes.sizeof(p))
        setattr(p, field, value)
        assert pe.lib.ewald_window_fit(ctypes.byref(p), 5, pe._ptr(z), pe._ptr(W), pe._ptr(DW)) == pe.EWALD_EINVAL
        assert pe.lib.ewald_radial_fit(ctypes.byref(p), 5, pe._ptr(r), pe._ptr(R), pe._ptr(G)) == pe.EWALD_EINVAL
        assert pe.lib.ewald_scale_table(ctypes.byref(p), pe._ptr(S)) == pe.EWALD_EINVAL, field
    assert pe.lib.ewald_window_fit(ctypes.byref(base), 5, pe._ptr(z), pe._ptr(W), pe._ptr(DW)) == pe.EWALD_OK


def test_null_arguments_are_rejected():
    """Every entry point that takes a plan, parameters or output pointers returns EWALD_EINVAL on NULL
    (before any CUDA call); destroying a NULL plan is a no-op."""
    import ctypes
    lib = pe.lib
    buf = np.zeros(16)
    cnt = ctypes.c_int(0)
    p = pe.ewald_params()
    calls = [lambda: lib.ewald_profile(None, 1),
             lambda: lib.ewald_profile_read(None, pe._ptr(buf), ctypes.byref(cnt)),
             lambda: lib.ewald_check(None, None),
             lambda: lib.ewald_debug_grid(None, 0, pe._ptr(buf)),
             lambda: lib.ewald_plan_query(None, None),
             lambda: lib.ewald_eval(None, None, None, None, None, None, None),
             lambda: lib.ewald_eval_host(None, None, None, None, None, None, None),
             lambda: lib.ewald_eval_batch(None, None, None, None, None, None, None, None),
             lambda: lib.ewald_plan_params_box(None, 100, ctypes.c_double(1e-6), None, ctypes.byref(p)),
             lambda: lib.ewald_plan_params(ctypes.c_double(1.0), 100, ctypes.c_double(1e-6), None, None),
             lambda: lib.ewald_opts_default(None),
             lambda: lib.ewald_window_fit(None, 0, None, None, None),
             lambda: lib.ewald_radial_fit(None, 0, None, None, None),
             lambda: lib.ewald_scale_table(None, None),
             lambda: lib.ewald_spread_static(None, None, None, None, None)]
    for k, call in enumerate(calls):
        assert call() == pe.EWALD_EINVAL, k
    lib.ewald_plan_destroy(None)


def test_static_spread_rejects_parameters_before_any_device_work():
    """ewald_spread_static checks its parameters before any CUDA call (the pointers below are never
    dereferenced): float32 (tile 8) parameters, a cuboid box, a window support out of range, no
    particles, and scratch beyond its static array."""
    import ctypes
    dummy = ctypes.c_void_p(16)

    def call(p):
        return pe.lib.ewald_spread_static(ctypes.byref(p), dummy, dummy, dummy, None), pe.lib.ewald_last_error()

    code, msg = call(pe.plan_params(1.0, 1000, 1e-6, precision="mixed"))
    assert code == pe.EWALD_EINVAL and b"tile 8" in msg
    code, msg = call(pe.plan_params((1.0, 1.0, 2.0), 1000, 1e-6))
    assert code == pe.EWALD_EINVAL and b"cubic" in msg
    for field, value in [("P", 30), ("n", 0), ("deg_w", 0)]:
        p = pe.plan_params(1.0, 1000, 1e-6)
        setattr(p, field, value)
        assert call(p)[0] == pe.EWALD_EINVAL, field
    code, msg = call(pe.plan_params(1.0, 10_000_000, 1e-8))
    assert code == pe.EWALD_ETOOBIG and b"static array" in msg


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
    assert o.autotune == 0 and o.grid_density == 0.0 and o.tol_safety == 0.25 and o.window_extra == 0
    o.autotune = 2
    p = pe.ewald_params()
    assert pe.lib.ewald_plan_params(1.0, 1000, 1e-6, ctypes.byref(o), ctypes.byref(p)) == pe.EWALD_EINVAL
    o = pe.make_opts()
    o.rc = float("nan")
    assert pe.lib.ewald_plan_params(1.0, 1000, 1e-6, ctypes.byref(o), ctypes.byref(p)) == pe.EWALD_EINVAL
    assert b"rc must be a number" in pe.lib.ewald_last_error()
    with pytest.raises(ValueError, match="precision must be one of"):
        pe.make_opts(precision="double")


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
def library_rule_box(Ls, n, tol, mult):
    """The cuboid reading (Alg. 3 in units of the shortest edge; oracle.params.plan_box) with the
    planner's additions (a)-(e); the cutoff fixed point uses the common spacing (V/(g n))^(1/3)."""
    Lv = np.asarray(Ls, dtype=np.float64)
    Lmin, V = float(Lv.min()), float(np.prod(Lv))
    t = tol * TOL_SAFETY

    def cutoff(t):
        r, h = 0.1, (V / (GRID_DENSITY[mult] * n)) ** (1.0 / 3.0)
        for _ in range(12):
            r = min(oparams.cs_of(r, t) * h / (math.pi * Lmin), 0.5)
        return r

    t_pot = t
    rcl = cutoff(t)
    m0 = oparams.cs_of(rcl, t) / (math.pi * rcl)
    if m0 > FORCE_M0:
        t *= FORCE_M0 / m0
        rcl = cutoff(t)
    cs = oparams.cs_of(rcl, t)
    ms = [good_size(math.ceil(cs * L / (math.pi * rcl * Lmin)), mult) for L in Lv]
    hmax = max(float(L) / m for L, m in zip(Lv, ms))
    rcl = cs * hmax / (math.pi * Lmin)
    cw = oparams.cw_of(oparams.cs_of(rcl, t_pot), rcl)
    P = int(math.ceil(2.0 * (rcl * cw / cs) * Lmin / hmax))
    return dict(m=ms, P=P, rc=rcl * Lmin, cs=cs, cw=math.pi * P / 2.0)


@pytest.mark.parametrize("box,n,tol,prec,mult", [((1.0, 1.25, 0.75), 5000, 1e-6, "fp64", 4),
                                                 ((1.0, 1.25, 0.75), 5000, 1e-6, "mixed", 8),
                                                 ((2.0, 1.0, 1.0), 100_000, 1e-10, "fp64", 4),
                                                 ((0.9, 1.7, 1.2), 40_000, 1e-8, "floatfloat", 4)])
def test_cuboid_plan_params_match_stated_rule(box, n, tol, prec, mult):
    p = pe.plan_params(box, n, tol, precision=prec)
    q = library_rule_box(box, n, tol, mult)
    assert list(p.grid) == q["m"] and p.P == q["P"] and p.deg_g > 0
    assert list(p.box) == list(box)
    for k in ("rc", "cs", "cw"):
        assert abs(getattr(p, k) / q[k] - 1) <= 1e-11, k
    for d in range(3):   # cells of edge >= rc / reach on every axis (z: rc / sr_reach_z)
        assert box[d] / p.cells[d] >= p.rc / (p.sr_reach_z if d == 2 else p.sr_reach) - 1e-15


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


def test_spread_kernel_choice():
    """ewald_opts.spread_kernel: 0 (automatic) and 1 give the CUDA-core kernel; 2 gives the tensor-core
    kernel only to float32 plans whose window support fits it (P <= 14); other values are rejected."""
    import ctypes
    for tol in (1e-4, 1e-6):
        assert pe.plan_params(1.0, 100_000, tol, precision="mixed").spread_kernel == 1
        assert pe.plan_params(1.0, 100_000, tol, precision="mixed", spread_kernel=1).spread_kernel == 1
        assert pe.plan_params(1.0, 100_000, tol, precision="mixed", spread_kernel=2).spread_kernel == 2
    for prec, tol in (("fp64", 1e-6), ("mixed", 1e-10), ("floatfloat", 1e-8)):
        p = pe.plan_params(1.0, 100_000, tol, precision=prec, spread_kernel=2)
        assert p.precision != pe.EWALD_MIXED and p.spread_kernel == 1
    p = pe.plan_params(1.0, 100_000, 1e-6, precision="mixed", spread_kernel=2, window_extra=3)
    assert p.P == 15 and p.spread_kernel == 1          # beyond the tensor-core kernel's accumulator
    o = pe.make_opts(precision="mixed")
    o.spread_kernel = 3
    q = pe.ewald_params()
    assert pe.lib.ewald_plan_params(1.0, 1000, 1e-6, ctypes.byref(o), ctypes.byref(q)) == pe.EWALD_EINVAL


def test_plan_create_without_a_device_reports_it():
    """On a host without a CUDA device, plan creation fails with EWALD_ECUDA naming the missing device
    (not as a failed allocation), after the argument checks, and leaves *out NULL."""
    import ctypes
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p(1)
    code = pe.lib.ewald_plan_create(ctypes.c_double(1.0), ctypes.c_int64(1000), ctypes.c_double(1e-6), None,
                                    ctypes.byref(h))
    assert code == pe.EWALD_ECUDA and b"no CUDA device" in pe.lib.ewald_last_error()
    assert h.value is None
    code = pe.lib.ewald_plan_create(ctypes.c_double(-1.0), ctypes.c_int64(1000), ctypes.c_double(1e-6), None,
                                    ctypes.byref(h))
    assert code == pe.EWALD_EINVAL
