"""Kernel splits for the Laplace kernel 1/r, plain FP64 (oracle; test use only).

PSWFSplit follows Sec. 4.1-4.2 of the paper:
  gamma_rc(x) = psi(x/rc) / (rc lambda_0 psi(0)) on [-rc, rc]        (eq. PSWF_mollifier)
  Phi(x)      = 2/(lambda_0 psi(0)) int_0^{x/rc} psi(u) du, x <= rc   (eq. Phi_cs)
  M(r)        = Phi(r)/r, R(r) = (1 - Phi(r))/r, R = 0 for r >= rc    (eq. M, eq. R)
  gammahat(w) = int gamma_rc(x) e^{-i w x} dx
              = 1/(lambda_0 psi(0)) int_{-1}^{1} psi(u) e^{-i w rc u} du
    (the definition in eq. gammahatintegral; its right-hand side as printed
    drops the 1/lambda_0 of gamma_rc, which eq. PSWF_mollifier_ft and
    gammahat(0) = int gamma = 1 restore)
  Mhat(w)     = 4 pi gammahat(|w|) / |w|^2                            (eq. MhatPSWF)
  self term   = -lim_{r->0} M(r) rho_i = -2 rho_i / (lambda_0 rc)     (Sec. 3.1, phi^self)
The self-term limit follows from Phi'(0) = 2 psi(0)/(lambda_0 psi(0)) = 2/lambda_0.

GaussianSplit is the classical Ewald split of Example 1 (Sec. 2.3):
  M = erf(r/sigma)/r, R = erfc(r/sigma)/r, Mhat = 4 pi/|w|^2 exp(-sigma^2 |w|^2 / 4),
  lim_{r->0} M(r) = 2/(sqrt(pi) sigma).

Parity status: pinned in tests/test_oracle_split.py (int gamma = 1, Phi(1) = 1,
R(rc) = 0, R >= 0, in-band gammahat equals psi(rc w/cs)/psi(0) by Lemma 2) and
through split independence of the total Ewald sum (tests/test_oracle_exact.py).
"""
import numpy as np
from scipy.special import erfc

from .pswf import PSWF


class PSWFSplit:
    """PSWF mollifier split with bandlimit cs and cutoff rc."""

    def __init__(self, cs, rc):
        self.cs = float(cs)
        self.rc = float(rc)
        self.f = PSWF(self.cs)
        self.norm = 2.0 / (self.f.lam * self.f.psi0)

    def gamma(self, x):
        x = np.abs(np.asarray(x, dtype=np.float64))
        inside = x <= self.rc
        u = np.where(inside, x / self.rc, 0.0)
        return np.where(inside, self.f.psi(u) / (self.rc * self.f.lam * self.f.psi0), 0.0)

    def Phi(self, r):
        r = np.asarray(r, dtype=np.float64)
        u = np.minimum(r / self.rc, 1.0)
        return np.where(r >= self.rc, 1.0, self.norm * self.f.int0(u))

    def dPhi(self, r):
        """d Phi / dr = 2 gamma_rc(r)."""
        return 2.0 * self.gamma(r)

    def R(self, r):
        r = np.asarray(r, dtype=np.float64)
        inside = r < self.rc
        rs = np.where(inside, r, 1.0)
        return np.where(inside, (1.0 - self.Phi(rs)) / rs, 0.0)

    def dR(self, r):
        """dR/dr = -(1 - Phi)/r^2 - Phi'(r)/r for r < rc, else 0."""
        r = np.asarray(r, dtype=np.float64)
        inside = r < self.rc
        rs = np.where(inside, r, 1.0)
        val = -(1.0 - self.Phi(rs)) / rs ** 2 - self.dPhi(rs) / rs
        return np.where(inside, val, 0.0)

    def R_and_dR(self, r):
        """R(r) and R'(r) for 0 < r < rc (one Phi evaluation)."""
        r = np.asarray(r, dtype=np.float64)
        one_m_phi = 1.0 - self.norm * self.f.int0(r / self.rc)
        return one_m_phi / r, -one_m_phi / r ** 2 - self.dPhi(r) / r

    def gammahat(self, omega):
        om = np.asarray(omega, dtype=np.float64) * self.rc
        return self.f.cos_transform(om) / (self.f.lam * self.f.psi0)

    def Mhat_k2(self, k2, L):
        """Mhat at integer |k|^2 (k != 0) of the box [0, L)^3: L^2/(pi |k|^2) gammahat(2 pi |k|/L)."""
        k2 = np.asarray(k2, dtype=np.float64)
        omega = 2.0 * np.pi * np.sqrt(k2) / L
        return L * L / (np.pi * k2) * self.gammahat(omega)

    def Mhat_w2(self, w2):
        """Mhat at |omega|^2 = w2 > 0 (any box shape): 4 pi / w2 * gammahat(sqrt(w2))."""
        w2 = np.asarray(w2, dtype=np.float64)
        return 4.0 * np.pi / w2 * self.gammahat(np.sqrt(w2))

    def self_coeff(self):
        return 2.0 / (self.f.lam * self.rc)


class GaussianSplit:
    """Classical Ewald split with Gaussian width sigma (Example 1)."""

    def __init__(self, sigma):
        self.sigma = float(sigma)

    def R(self, r):
        r = np.asarray(r, dtype=np.float64)
        return erfc(r / self.sigma) / r

    def dR(self, r):
        r = np.asarray(r, dtype=np.float64)
        s = self.sigma
        return -erfc(r / s) / r ** 2 - 2.0 / (np.sqrt(np.pi) * s) * np.exp(-(r / s) ** 2) / r

    def R_and_dR(self, r):
        return self.R(r), self.dR(r)

    def Mhat_k2(self, k2, L):
        k2 = np.asarray(k2, dtype=np.float64)
        omega2 = (2.0 * np.pi / L) ** 2 * k2
        return 4.0 * np.pi / omega2 * np.exp(-self.sigma ** 2 * omega2 / 4.0)

    def Mhat_w2(self, w2):
        w2 = np.asarray(w2, dtype=np.float64)
        return 4.0 * np.pi / w2 * np.exp(-self.sigma ** 2 * w2 / 4.0)

    def self_coeff(self):
        return 2.0 / (np.sqrt(np.pi) * self.sigma)
