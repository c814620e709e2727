"""Pins of the oracle's step-by-step Alg. 2 and of the Alg. 3 parameters (Secs. 3.2, 5, 6)."""
import math

import numpy as np
import pytest
from scipy.special import lambertw

from oracle import exact, params
from oracle.alg2 import Alg2
from oracle.pswf import PSWF
from paper_2602_16591_gb300.workloads import uniform_alternating, uniform_neutral


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
def test_alg2_meets_tolerance(tol):
    """E8: the fast method with Alg. 3 parameters meets the requested relative tolerance."""
    x, rho, L = uniform_alternating(1000, seed=0)
    p = params.plan(L, len(x), tol, tol_safety=0.25)
    ref = exact.pswf_exact(x, rho, L)
    A = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"])
    out = A.total(x, rho)
    assert _rel(out[0], ref[0]) <= 2 * tol
    assert _rel(out[3], ref[3]) <= 2 * tol
    assert abs(out[2] - ref[2]) <= 2 * tol * abs(ref[2])


def test_cube_corners_are_unstable_ball_is_not():
    """Deconvolving the corners of I_m amplifies rounding (reading recorded in the design doc)."""
    x, rho, L = uniform_neutral(1500, seed=1)
    p = params.plan(L, len(x), 1e-8, tol_safety=0.25)
    ref = exact.pswf_exact(x, rho, L)
    cube = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"], ball=False).total(x, rho)
    ball = Alg2(L, p["m"], p["P"], p["cs"], p["cw"], p["rc"], ball=True).total(x, rho)
    assert _rel(ball[0], ref[0]) <= 2e-8
    assert _rel(cube[0], ref[0]) > 1e3 * _rel(ball[0], ref[0])


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
    for n, tol in [(1000, 1e-6), (100_000, 1e-6), (100_000, 1e-10), (10_000_000, 1e-8)]:
        p = params.plan(1.0, n, tol)
        m = p["m"]
        r = m
        for q in (2, 3, 5, 7):
            while r % q == 0:
                r //= q
        assert r == 1 and m % 4 == 0
        assert abs(p["cs"] / p["rc"] - math.pi * m / p["L"]) < 1e-9 * p["cs"] / p["rc"]
        assert abs(p["cs"] / p["rc"] - p["cw"] / p["alpha"]) < 1e-9 * p["cs"] / p["rc"]
        assert p["P"] == math.ceil(2 * p["cw_target"] / math.pi - 1e-12)
        assert p["rc"] <= 0.5 * p["L"]


def test_kappa_against_direct_sum():
    K = 40
    r = np.arange(-K, K + 1)
    k2 = (r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2).ravel()
    k2 = k2[(k2 > 0) & (k2 <= K * K)].astype(float)
    direct = np.sum(1.0 / k2 ** 2) + 4 * math.pi / K
    assert abs(direct / math.pi ** 2 / params.KAPPA - 1) < 2e-3


def test_lambertw_branches():
    z = -2 * params.KAPPA * 1e-12 / params.A_W ** 2
    w = float(np.real(lambertw(z, -1)))
    assert w < -1 and abs(w * math.exp(w) / z - 1) < 1e-12


# ------------------------------------------------------------------ cuboid boxes (Remark, Sec. 6.1) --
def test_cuboid_alg2_supercell_equals_cube():
    """Alg. 2 on a 1x1x2 supercell grid (m, m, 2m) is the cube's Alg. 2 for every copy (same discrete
    operators: the spread grid and the scaled modes of the supercell are those of the cube interleaved)."""
    from oracle import params as op
    rng = np.random.default_rng(7)
    x = rng.random((60, 3))
    q = rng.uniform(-1, 1, 60)
    q -= q.mean()
    p = op.plan(1.0, 60, 1e-6, grid_density=8.0)
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
    """The cuboid plan rule (oracle params.plan_box) meets tol against the converged cuboid sum."""
    from oracle import params as op
    Lv = (1.0, 1.25, 0.75)
    rng = np.random.default_rng(8)
    x = rng.random((400, 3)) * np.array(Lv)
    q = rng.uniform(-1, 1, 400)
    q -= q.mean()
    p = op.plan_box(Lv, 400, tol, grid_density=3.0, tol_safety=0.25)
    assert len(set(p["m"])) >= 2          # a genuinely anisotropic grid
    A = Alg2(Lv, p["m"], p["P"], p["cs"], p["cw"], p["rc"])
    phi, grad, E, F = A.total(x, q)
    ref = exact.pswf_exact(x, q, Lv)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert rel(phi, ref[0]) <= tol
    assert rel(F, ref[3]) <= 2 * tol


def test_cuboid_plan_reduces_to_cube():
    from oracle import params as op
    for tol in (1e-4, 1e-8):
        a = op.plan(1.3, 5000, tol, grid_density=3.0, tol_safety=0.25)
        b = op.plan_box((1.3, 1.3, 1.3), 5000, tol, grid_density=3.0, tol_safety=0.25)
        assert b["m"] == [a["m"]] * 3 and b["P"] == a["P"] and b["rc"] == a["rc"]
