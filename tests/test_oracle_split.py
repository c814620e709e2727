"""Pins of the oracle's kernel split (Sec. 4.1-4.2, Table 1, Remarks on Phi and R)."""
import numpy as np
import pytest
from scipy.special import erfc

from oracle.pswf import gauss_legendre
from oracle.split import GaussianSplit, PSWFSplit

CASES = [(8.0, 0.1), (14.0, 0.3), (25.0, 0.5)]


@pytest.mark.parametrize("cs,rc", CASES)
def test_mollifier_integrates_to_one(cs, rc):
    sp = PSWFSplit(cs, rc)
    t, w = gauss_legendre(200)
    assert abs(rc * np.sum(w * sp.gamma(rc * t)) - 1.0) <= 1e-13
    assert abs(sp.gammahat(0.0) - 1.0) <= 1e-13


@pytest.mark.parametrize("cs,rc", CASES)
def test_phi_and_r_compact_support(cs, rc):
    """Phi(rc) = 1, R(rc) = 0, R >= 0, Phi nondecreasing (Remarks in Sec. 4.1)."""
    sp = PSWFSplit(cs, rc)
    assert abs(sp.Phi(np.array([rc]))[0] - 1.0) <= 1e-13
    r = np.linspace(1e-3 * rc, rc * (1 - 1e-12), 500)
    R = sp.R(r)
    assert np.all(R >= -1e-14)
    assert abs(sp.R(np.array([rc * (1 - 1e-9)]))[0]) <= 1e-6 / rc
    assert np.all(sp.R(np.array([rc, 1.5 * rc])) == 0.0)
    assert np.all(np.diff(sp.Phi(r)) >= -1e-15)


@pytest.mark.parametrize("cs,rc", CASES)
def test_split_sums_to_coulomb(cs, rc):
    """M + R = 1/r with M = Phi/r."""
    sp = PSWFSplit(cs, rc)
    r = np.linspace(0.01 * rc, 2 * rc, 50)
    assert np.allclose(sp.Phi(r) / r + sp.R(r), 1.0 / r, rtol=1e-14, atol=0)


@pytest.mark.parametrize("cs,rc", CASES)
def test_dR_matches_finite_difference(cs, rc):
    sp = PSWFSplit(cs, rc)
    r = np.linspace(0.05 * rc, 0.95 * rc, 19)
    h = 1e-6 * rc
    fd = (sp.R(r + h) - sp.R(r - h)) / (2 * h)
    assert np.allclose(sp.dR(r), fd, rtol=1e-7, atol=1e-7 / rc ** 2)


@pytest.mark.parametrize("cs,rc", CASES)
def test_gammahat_in_band_equals_psi(cs, rc):
    """eq. PSWF_mollifier_ft: gammahat(w) = psi(rc w / cs)/psi(0) for |w| <= cs/rc (Lemma 2)."""
    sp = PSWFSplit(cs, rc)
    w = np.linspace(0.0, cs / rc, 23)
    assert np.allclose(sp.gammahat(w), sp.f.psi(rc * w / cs) / sp.f.psi0, rtol=0, atol=1e-13)


def test_self_coefficient_is_limit_of_M():
    sp = PSWFSplit(14.0, 0.2)
    r = 1e-7
    assert abs(sp.Phi(np.array([r]))[0] / r - sp.self_coeff()) <= 1e-6 * sp.self_coeff()


def test_gaussian_split_closed_forms():
    g = GaussianSplit(0.1)
    r = np.array([0.05, 0.1, 0.3])
    assert np.allclose(g.R(r), erfc(r / 0.1) / r, rtol=1e-15)
    # Mhat at small k tends to 4 pi/w^2
    L = 1.0
    k2 = np.array([1.0])
    w2 = (2 * np.pi) ** 2
    assert abs(g.Mhat_k2(k2, L)[0] - 4 * np.pi / w2 * np.exp(-0.01 * w2 / 4)) < 1e-15
