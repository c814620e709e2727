"""First prolate spheroidal wave function psi_0^c, plain FP64 (oracle; test use only).

Follows the paper's Sec. 2.4 and App. B:

* psi_0^c is the eigenfunction, smallest eigenvalue chi_0, of the Sturm-Liouville
  ODE (1-s^2) psi'' - 2 s psi' + (chi_0 - c^2 s^2) psi = 0  (eq. ode), expanded in
  even Legendre polynomials psi = sum_k a_2k P_2k  (eq. PSWFLegendre).
* The operator -(d/ds)(1-s^2)(d/ds) + c^2 s^2 is diagonal + c^2 (s^2) in the
  orthonormal Legendre basis Pbar_k = sqrt(k+1/2) P_k.  Here the s^2 block is
  built as the square of the textbook Jacobi matrix of x P_k (three-term
  recurrence) and the eigenproblem is solved by a *dense* symmetric solver
  (numpy.linalg.eigh) -- deliberately a different route from the
  Sturm-bisection + inverse-iteration solver of the CUDA library's planner.
* Normalisation ||psi||_{L2[-1,1]} = 1 and psi(0) > 0 (Sec. 2.4).
* lambda_0 = (1/psi(0)) int_{-1}^{1} psi (App. B, "Evaluation of psi and lambda_0").
* Outside [-1,1] psi is continued through the eigen-relation
  lambda_0 psi(s) = int_{-1}^{1} psi(t) e^{i c s t} dt  (eq. eigenvalueproblem).

Parity status: pinned (tests/test_oracle_pswf.py) by Lemma 2, the ODE residual,
scipy.special.pro_cv / pro_ang1, Lemma 3 (chi_0 <= c^2/3), Lemma 4 (tail bound)
and the Table 5 curve fits.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(npts):
    """Gauss-Legendre nodes and weights on [-1, 1] (library routine)."""
    return npleg.leggauss(int(npts))


class PSWF:
    """psi_0^c on [-1, 1] from its Legendre expansion (App. B)."""

    def __init__(self, c, nterms=None):
        c = float(c)
        if c <= 0:
            raise ValueError("bandlimit c must be positive")
        self.c = c
        # number of even Legendre terms; App. B: K ~ 1.2 c suffices for 1e-12, add margin
        K = int(nterms) if nterms else int(np.ceil(1.2 * c)) + 24
        self.nterms = K
        N = 2 * K + 2
        j = np.arange(N - 1, dtype=np.float64)
        # x P_j = ((j+1) P_{j+1} + j P_{j-1}) / (2j+1)  ->  orthonormal Jacobi matrix
        off = (j + 1.0) / np.sqrt((2.0 * j + 1.0) * (2.0 * j + 3.0))
        J = np.diag(off, 1) + np.diag(off, -1)
        S2 = J @ J                              # multiplication by s^2
        ev = 2 * np.arange(K)                   # even degrees 0, 2, ..., 2K-2
        A = np.diag(ev * (ev + 1.0)) + c * c * S2[np.ix_(ev, ev)]
        w, V = np.linalg.eigh(A)
        self.chi = float(w[0])
        v = V[:, 0]
        a = np.zeros(2 * K - 1)
        a[ev] = v * np.sqrt(ev + 0.5)           # standard (unnormalised) Legendre coefficients
        if npleg.legval(0.0, a) < 0:
            a = -a
        self.a = a
        self.da = npleg.legder(a)
        self.ia = npleg.legint(a, lbnd=0)       # antiderivative vanishing at 0
        self.psi0 = float(npleg.legval(0.0, a))
        self.lam = float(2.0 * a[0] / self.psi0)  # int_{-1}^{1} P_0 = 2, the other P_2k integrate to 0
        self.psi1 = float(npleg.legval(1.0, a))

    # --- evaluation on [-1, 1] -------------------------------------------------
    def psi(self, x):
        """psi_0^c(x) for |x| <= 1 (Legendre series)."""
        return npleg.legval(np.asarray(x, dtype=np.float64), self.a)

    def dpsi(self, x):
        """(psi_0^c)'(x) for |x| <= 1 (differentiated Legendre series, App. B)."""
        return npleg.legval(np.asarray(x, dtype=np.float64), self.da)

    def int0(self, x):
        """int_0^x psi_0^c(u) du for |x| <= 1."""
        return npleg.legval(np.asarray(x, dtype=np.float64), self.ia)

    # --- Fourier side -------------------------------------------------------------
    def cos_transform(self, omega):
        """int_{-1}^{1} psi(u) cos(omega u) du, any real omega (Gauss-Legendre)."""
        om = np.atleast_1d(np.asarray(omega, dtype=np.float64))
        npts = self.nterms + int(0.6 * np.max(np.abs(om))) + 48
        t, wt = gauss_legendre(npts)
        pw = self.psi(t) * wt
        out = np.cos(np.outer(om, t)) @ pw
        return out.reshape(np.shape(omega)) if np.ndim(omega) else float(out[0])

    def psi_ext(self, s):
        """psi_0^c(s) for any real s, continued by the eigen-relation (eq. eigenvalueproblem)."""
        s = np.asarray(s, dtype=np.float64)
        return self.cos_transform(self.c * s) / self.lam
