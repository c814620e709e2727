"""Pins of the oracle's step-by-step Alg. 2 and of the Alg. 3 parameters (Secs. 3.2, 5, 6)."""
import math

import numpy as np
import pytest

from oracle import exact, params
from oracle.alg2 import Alg2
from oracle.pswf import PSWF
from workloads import uniform_alternating, uniform_neutral


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def test_single_charge_dft_is_window_transform():
    """DFT of one spread charge: |ahat_k| h^3 = phihat(k) up to aliasing (Poisson summation)."""
    L, m, P = 1.0, 16, 12
    A = Alg2(L, m, P, cs=10.0, cw=math.pi * P / 2, rc=10.0 / (math.pi * m))
    x = np.array([[0.3137, 0.5519, 0.0803]])
    a = A.spread(x, np.array([1.0]))
    ah = A.fft(a)
    k = A.kgrid()
    h = L / m
    ph1 = A.alpha * A.win.cos_transform(2 * np.pi * k / L * A.alpha) / A.win.psi0 / h
    main = ph1[:, None, None] * ph1[None, :, None] * ph1[None, None, :]
    lo = (np.abs(k) <= m // 4)
    sel = lo[:, None, None] & lo[None, :, None] & lo[None, None, :]
    # aliases are bounded by psi(1)/psi(0) ~ 2e-7 at c_w = 6 pi (Lemma 4, Table 5)
    assert np.max(np.abs(np.abs(ah[sel]) - main[sel]) / main[sel]) < 2e-6


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
@pytest.mark.parametrize("rc", [0.2, 0.3])
def test_alg2_meets_tolerance(tol, rc):
    """Alg. 3 as printed (with the relative-tolerance reading) gives an error close to tol (Remark after
    Alg. 3): potential and energy within 2 tol of the converged sum.  The paper has no force model;
    the forces are bounded loosely here and pinned exactly elsewhere (gradient = -F)."""
    x, rho, L = uniform_alternating(1000, seed=0)
    p = params.plan(L, tol, rc)
    ref = exact.pswf_exact(x, rho, L)
    A = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"])
    out = A.total(x, rho)
    assert 0.3 * tol <= _rel(out[0], ref[0]) <= 2 * tol     # near tol, not far below it
    assert abs(out[2] - ref[2]) <= 4 * tol * abs(ref[2])
    assert _rel(out[3], ref[3]) <= 10 * tol


@pytest.mark.parametrize("tol", [1e-3, 1e-4])
def test_cube_of_alg2_agrees_with_band_where_stable(tol):
    """Alg. 2 as printed scales every mode of the cube I_m.  Where that is numerically stable (loose
    tolerances) it agrees with the band-limited reading within the tolerance, and both meet it."""
    x, rho, L = uniform_neutral(1500, seed=1)
    ref = exact.pswf_exact(x, rho, L)
    for rc in (0.15, 0.25):
        p = params.plan(L, tol, rc)
        cube = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"], modes="cube").total(x, rho)
        band = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"]).total(x, rho)
        assert _rel(cube[0], ref[0]) <= 2 * tol
        assert _rel(band[0], ref[0]) <= 2 * tol
        assert _rel(cube[0], band[0]) <= 2 * tol


def test_cube_corners_are_unstable_band_is_not():
    """Deconvolving the corners of I_m amplifies rounding: the whole cube of Alg. 2 as printed loses
    every digit at tol 1e-8, the modes inside the mollifier's band do not."""
    x, rho, L = uniform_neutral(1500, seed=1)
    p = params.plan(L, 1e-8, 0.2)
    ref = exact.pswf_exact(x, rho, L)
    cube = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"], modes="cube").total(x, rho)
    band = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"], modes="band").total(x, rho)
    assert _rel(band[0], ref[0]) <= 2e-8
    assert _rel(cube[0], ref[0]) > 1e3 * _rel(band[0], ref[0])


def test_error_models_match_measured_split_error():
    """Fig. 5-style check: measured absolute RMS error of the far field vs the closed-form
    split model (eq. PSWF_model, A_s = 5) when the window error is negligible."""
    x, rho, L = uniform_neutral(400, seed=5, dist="normal")
    rc = 0.1
    ref = exact.pswf_exact(x, rho, L)
    for m in (24, 36):
        cs = math.pi * rc * m / L
        P = 24
        A = Alg2(L, m, P, cs, math.pi * P / 2, rc)
        out = A.total(x, rho)
        err = np.sqrt(np.mean((out[0] - ref[0]) ** 2))
        model = 5.0 * np.linalg.norm(rho) / math.sqrt(L ** 3) * math.sqrt(rc) * cs ** -0.5 * math.exp(-cs)
        assert model / 4 <= err <= model * 4, (m, err, model)


def test_split_error_grows_as_sqrt_rc_at_fixed_cs():
    """Fig. 6 and Prop. 1: with c_s held fixed (c_s = pi r_c m / L = 4 pi, so m = 64, 32, 16 for
    r_c = L/16, L/8, L/4) and the window error negligible (P = 16), the far-field error grows as
    sqrt(r_c): the least-squares slope of log(err) on log(r_c) is 1/2 within 0.1, and every error is
    within [0.7, 1.4] of eq. PSWF_model with A_s = 5 (a model in r_c or without r_c gives slope 1 or 0)."""
    x, rho, L = uniform_neutral(400, seed=5, dist="normal")
    ref = exact.pswf_exact(x, rho, L)
    rcs, errs = [], []
    for rc, m in ((0.0625, 64), (0.125, 32), (0.25, 16)):
        cs = math.pi * rc * m / L
        P = 16
        out = Alg2(L, m, P, cs, math.pi * P / 2, rc).total(x, rho)
        err = np.sqrt(np.mean((out[0] - ref[0]) ** 2))
        model = 5.0 * np.linalg.norm(rho) / math.sqrt(L ** 3) * math.sqrt(rc) * cs ** -0.5 * math.exp(-cs)
        assert 0.7 <= err / model <= 1.4, (rc, err, model)
        rcs.append(rc)
        errs.append(err)
    slope = np.polyfit(np.log(rcs), np.log(errs), 1)[0]
    assert abs(slope - 0.5) <= 0.1, slope


def test_alg2_scaling_law_and_a_planted_unit_mistake():
    """eq. phinondim for Alg. 2 itself: scaling the box, the positions and the cutoff by s with the same
    (m, P, c_s, c_w) divides phi by s and F by s^2 to rounding, since the grid spacing, alpha, the
    window transform per h and the 1/V of the scaling all carry their units.  Every other cube test of
    Alg. 2 runs at L = 1, where a dropped 1/V is invisible; planted here, it breaks the law."""
    x, rho, L = uniform_neutral(300, seed=8)
    m, P, rc, s = 24, 12, 0.2, 2.5
    cs, cw = math.pi * rc * m / L, math.pi * P / 2
    a = Alg2(L, m, P, cs, cw, rc).total(x, rho)
    b = Alg2(s * L, m, P, cs, cw, s * rc).total(s * x, rho)
    assert _rel(b[0], a[0] / s) <= 1e-12
    assert _rel(b[3], a[3] / s ** 2) <= 1e-12

    class NoVolume(Alg2):   # the planted mistake: S(k) without its 1/V
        def scaling(self):
            return super().scaling() * float(np.prod(self.Lv))

    a2 = NoVolume(L, m, P, cs, cw, rc).total(x, rho)
    b2 = NoVolume(s * L, m, P, cs, cw, s * rc).total(s * x, rho)
    assert _rel(a2[0], a[0]) <= 1e-14                  # invisible at L = 1
    assert _rel(b2[0], a2[0] / s) > 0.1


def test_alias_model_matches_measured_window_error():
    """Fig. 5(a)-style: with a large m the error plateau follows eq. window_err_model (A_w = 3.1)."""
    x, rho, L = uniform_neutral(400, seed=6, dist="normal")
    ref = exact.pswf_exact(x, rho, L)
    m = 40
    rc = 0.4
    cs = math.pi * rc * m / L
    for P in (6, 8):
        cw = math.pi * P / 2
        out = Alg2(L, m, P, cs, cw, rc).total(x, rho)
        err = np.sqrt(np.mean((out[0] - ref[0]) ** 2))
        model = 3.1 * np.linalg.norm(rho) / math.sqrt(L ** 3) * math.sqrt(L) * cw ** 0.5 * math.exp(-cw)
        assert model / 4 <= err <= model * 4, (P, err, model)


def test_params_lambert_equations():
    """Alg. 3 steps 1-2: c_s solves 2 c_s e^{2 c_s} = 2 (B_s/eps)^2; c_w balances the models."""
    for tol in (1e-4, 1e-6, 1e-10):
        rcl = 0.08
        cs = params.cs_of(rcl, tol)
        bs_eps = params.A_S * math.sqrt(rcl) / (math.sqrt(params.KAPPA) * tol)
        assert abs(2 * cs * math.exp(2 * cs) / (2 * bs_eps ** 2) - 1) < 1e-12
        cw = params.cw_of(cs, rcl)
        lhs = params.A_W * cw ** 0.5 * math.exp(-cw)
        rhs = params.A_S * math.sqrt(rcl) * cs ** -0.5 * math.exp(-cs)
        assert abs(lhs / rhs - 1) < 1e-10
        assert cw > 1.0   # large root of the W_{-1} branch


def test_params_structure():
    """Alg. 3 steps 3-5 and the instantiation reading: eq. csrc and eq. bandwidth hold exactly after
    rounding, P follows eq. P_dimless from the unrounded window, c_w = pi P/2 (eq. cwP)."""
    for tol, rc in [(1e-4, 0.1), (1e-6, 0.05), (1e-10, 0.2), (1e-8, 0.026)]:
        q = params.alg3(1.0, tol, rc)
        assert q["m"] == math.ceil(q["cs"] / (math.pi * rc))
        assert q["P"] == math.ceil(2 * q["alpha"] * q["m"])
        assert abs(q["alpha"] - rc * q["cw"] / q["cs"]) < 1e-15
        p = params.plan(1.0, tol, rc)
        assert p["m"] % 2 == 0 and q["m"] <= p["m"] <= q["m"] + 1
        assert abs(p["cs"] / p["rc"] - math.pi * p["m"] / p["L"]) < 1e-12 * p["cs"] / p["rc"]
        assert abs(p["cs"] / p["rc"] - p["cw"] / p["alpha"]) < 1e-12 * p["cs"] / p["rc"]
        assert p["P"] == math.ceil(2 * (rc * q["cw"] / q["cs"]) * p["m"] - 1e-12)
        assert p["rc"] <= rc and abs(p["cw"] - math.pi * p["P"] / 2) < 1e-15


def test_alg3_worked_numbers():
    """Numbers the paper states about Alg. 3: A_s/A_w = 4 sqrt(5)/pi^(3/2) ~ 1.61 (Sec. 6.3), and with
    c_s = log(1/eps) and r_c = 0.1 (Table 3's setting) steps 4-5 give the bandlimit-sized m, i.e. within
    a few modes of the smallest m Table 3 reports (42 at 1e-6, 72 at 1e-10)."""
    assert abs(params.A_S / params.A_W - 4 * math.sqrt(5) / math.pi ** 1.5) < 0.01
    for eps, m_table in ((1e-6, 42), (1e-10, 72)):
        q = params.alg3(1.0, eps, 0.1, cs=math.log(1 / eps))
        assert m_table <= q["m"] <= m_table + 3


# ------------------------------------------------------------------ cuboid boxes (Remark, Sec. 6.1) --
def test_cuboid_alg2_supercell_equals_cube():
    """Alg. 2 on a 1x1x2 supercell grid (m, m, 2m) is the cube's Alg. 2 for every copy (same discrete
    operators: the spread grid and the scaled modes of the supercell are those of the cube interleaved)."""
    from oracle import params as op
    rng = np.random.default_rng(7)
    x = rng.random((60, 3))
    q = rng.uniform(-1, 1, 60)
    q -= q.mean()
    p = op.plan(1.0, 1e-6, 0.35)
    A = Alg2(1.0, p["m"], p["P"], p["cs"], p["cw"], p["rc"])
    phi, grad, E, F = A.total(x, q)
    B = Alg2((1.0, 1.0, 2.0), (p["m"], p["m"], 2 * p["m"]), p["P"], p["cs"], p["cw"], p["rc"])
    xs = np.concatenate([x, x + np.array([0.0, 0.0, 1.0])])
    phis, grads, Es, Fs = B.total(xs, np.tile(q, 2))
    for c in range(2):
        assert np.max(np.abs(phis[c * 60:(c + 1) * 60] - phi)) <= 1e-12 * np.max(np.abs(phi))
        assert np.max(np.abs(Fs[c * 60:(c + 1) * 60] - F)) <= 1e-11 * np.max(np.abs(F))
    assert abs(Es - 2 * E) <= 1e-12 * abs(2 * E)


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
def test_cuboid_alg2_meets_tolerance(tol):
    """Alg. 3 for a cuboid (reading: units of the shortest edge) meets tol against the converged sum."""
    from oracle import params as op
    Lv = (1.0, 1.25, 0.75)
    rng = np.random.default_rng(8)
    x = rng.random((400, 3)) * np.array(Lv)
    q = rng.uniform(-1, 1, 400)
    q -= q.mean()
    p = op.plan_box(Lv, tol, 0.3)
    assert len(set(p["m"])) >= 2          # a genuinely anisotropic grid
    A = Alg2(Lv, p["m"], p["P"], p["cs"], p["cw"], p["rc"])
    phi, grad, E, F = A.total(x, q)
    ref = exact.pswf_exact(x, q, Lv)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert rel(phi, ref[0]) <= 2 * tol
    assert rel(F, ref[3]) <= 10 * tol


def test_cuboid_plan_reduces_to_cube():
    from oracle import params as op
    for tol in (1e-4, 1e-8):
        a = op.plan(1.3, tol, 0.2)
        b = op.plan_box((1.3, 1.3, 1.3), tol, 0.2)
        assert b["m"] == [a["m"]] * 3 and b["P"] == a["P"] and b["rc"] == a["rc"]
