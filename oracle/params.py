"""Alg. 3 parameter selection (Sec. 6), plain FP64 with scipy's Lambert W (oracle; test use only).

Steps of Alg. 3 with the readings the library uses (all recorded in the design doc):

* Relative tolerance.  Alg. 3 targets an absolute RMS error eps.  A relative
  tolerance tol is mapped to eps = tol * sqrt(kappa) ||rho||_2 / L, where
  kappa = pi^-2 sum_{k != 0} |k|^-4 is the mean square of the neutralised periodic
  potential of unit-norm uniform charges (Parseval with c_k = Mhat/V, eq. fcoeffs).
  Then B_s/eps = A_s sqrt(rc/L) / (sqrt(kappa) tol) needs no rho (Sec. 6.2).
* c_s = W_0(2 (B_s/eps)^2)/2       (eq. cs_dimless, principal branch: argument > 0)
* c_w = -W_{-1}(-2 B_w^2 e^{-2 c_s}/c_s)/2, B_w = (A_s/A_w) sqrt(rc/L)
                                   (eq. cwW, lower branch: the large root)
* rc (Sec. 6.2.2 leaves it to tuning): fixed point rc = c_s(rc) L / (pi (g n)^{1/3})
  for grid density g = m^3/n, capped at L/2 so the minimum image is exact.
* m = ceil(L c_s/(pi rc)) (eq. m_cs_dimless), rounded up to a multiple of 4 that
  has no prime factor above 7; then rc := c_s L/(pi m) so eq. csrc holds exactly.
* alpha = rc c_w/c_s, P = ceil(2 alpha m/L) (eqs. alpha, P_dimless); with the rc
  above this equals ceil(2 c_w/pi).  The window is instantiated with
  c_w := pi P/2 and alpha := P h/2 (eq. cwP), so c_s/rc = c_w/alpha (eq. bandwidth).
* Forces (no model in the paper): measured relative force errors are ~m/10 times the
  potential errors and follow the split truncation (c_s), not the window, so the split
  target tol*tol_safety is multiplied by min(1, 10/m0), m0 = c_s/(pi rc/L) before rounding,
  and rc re-derived; c_w (the window) is balanced against the untightened target.

Parity status: pinned in tests/test_oracle_params.py (Lambert-W identities,
balance equation eq. cwcs_model_dimless, kappa against a direct lattice sum).
"""
import math

import numpy as np
from scipy.special import lambertw

A_S = 5.0      # Sec. 5.1.1: fitted split-model prefactor
A_W = 3.1      # Sec. 5.2.1: fitted aliasing-model prefactor


def lattice_sum_k4(nmax=40000):
    """sum_{k in Z^3 \\ 0} |k|^-4 = sum_n r3(n)/n^2 with the tail sum_{n>N} ~ 4 pi/sqrt(N)."""
    K = int(math.isqrt(nmax)) + 1
    r = np.arange(-K, K + 1)
    sq = r * r
    n2 = (sq[:, None, None] + sq[None, :, None] + sq[None, None, :]).ravel()
    n2 = n2[(n2 > 0) & (n2 <= nmax)].astype(np.float64)
    s = float(np.sum(1.0 / n2 ** 2))
    # mean density of representations: r3(n) ~ 2 pi sqrt(n); tail integral from nmax + 1/2
    return s + 4.0 * math.pi / math.sqrt(nmax + 0.5)


KAPPA = lattice_sum_k4() / math.pi ** 2


def good_size(m, mult=4):
    """Smallest m' >= m, m' % mult == 0, with prime factors in {2, 3, 5, 7}."""
    m = max(int(m), mult)
    while True:
        if m % mult == 0:
            r = m
            for p in (2, 3, 5, 7):
                while r % p == 0:
                    r //= p
            if r == 1:
                return m
        m += 1


def cs_of(rc_over_L, tol):
    bs_eps = A_S * math.sqrt(rc_over_L) / (math.sqrt(KAPPA) * tol)
    return 0.5 * float(np.real(lambertw(2.0 * bs_eps ** 2, 0)))


def cw_of(cs, rc_over_L):
    bw = (A_S / A_W) * math.sqrt(rc_over_L)
    z = -2.0 * bw * bw * math.exp(-2.0 * cs) / cs
    return -0.5 * float(np.real(lambertw(z, -1)))


def plan(L, n, tol, grid_density=1.0, rc=None, tol_safety=1.0, mult=4):
    """Alg. 3 with the readings above; returns a dict of plan parameters.

    ``mult`` is the multiple m is rounded to (the library's spreading tile edge: 8 for its float32
    plans, 4 otherwise); the paper only needs an even, FFT-friendly m.
    """
    t = tol * tol_safety

    def cutoff(t):
        if rc is None:
            mstar = (grid_density * n) ** (1.0 / 3.0)
            r = 0.1
            for _ in range(12):
                r = min(cs_of(r, t) / (math.pi * mstar), 0.5)
            return r
        return min(rc / L, 0.5)

    t_pot = t
    rcl = cutoff(t)
    m0 = cs_of(rcl, t) / (math.pi * rcl)
    if m0 > 10.0:
        t *= 10.0 / m0
        rcl = cutoff(t)
    cs = cs_of(rcl, t)
    m = good_size(math.ceil(cs / (math.pi * rcl)), mult)
    rcl = cs / (math.pi * m)
    cw = cw_of(cs_of(rcl, t_pot), rcl)      # window balanced against the potential target
    alpha_over_L = rcl * cw / cs
    P = int(math.ceil(2.0 * alpha_over_L * m))
    h = L / m
    return dict(L=L, rc=rcl * L, cs=cs, cw_target=cw, cw=math.pi * P / 2.0, m=m, P=P,
                h=h, alpha=P * h / 2.0)


def plan_box(Ls, n, tol, grid_density=1.0, rc=None, tol_safety=1.0, mult=4):
    """Alg. 3 for a cuboid box (Remark on cuboid domains, Sec. 6.1).

    The parameters are derived in units of L_min = min_d L_d (the nondimensionalisation of the
    Remark): r_c/L_min and the Lambert-W equations as for a cube of edge L_min; the cutoff rule uses
    the common target spacing h = (V/(g n))^{1/3}.  Each axis gets m_d = ceil(c_s L_d/(pi r_c)),
    rounded as in ``plan``; then r_c := c_s h_max/pi with h_max = max_d L_d/m_d (eq. csrc on the
    coarsest axis; the other axes resolve more modes than the retained ellipsoid uses), and
    P = ceil(2 alpha/h_max) with alpha = r_c c_w/c_s, i.e. P = ceil(2 c_w/pi), instantiated with
    c_w := pi P/2 and alpha_d := P h_d/2 per axis.  A cube gives exactly ``plan``.
    """
    Lv = np.broadcast_to(np.asarray(Ls, dtype=np.float64), (3,))
    if np.all(Lv == Lv[0]):
        q = plan(float(Lv[0]), n, tol, grid_density=grid_density, rc=rc, tol_safety=tol_safety, mult=mult)
        q.update(m=[q["m"]] * 3, h=[q["h"]] * 3, alpha=[q["alpha"]] * 3, L=[q["L"]] * 3)
        return q
    Lmin, V = float(np.min(Lv)), float(np.prod(Lv))
    t = tol * tol_safety

    def cutoff(t):
        if rc is None:
            h = (V / (grid_density * n)) ** (1.0 / 3.0)
            r = 0.1
            for _ in range(12):
                r = min(cs_of(r, t) * h / (math.pi * Lmin), 0.5)
            return r
        return min(rc / Lmin, 0.5)

    t_pot = t
    rcl = cutoff(t)
    m0 = cs_of(rcl, t) / (math.pi * rcl)
    if m0 > 10.0:
        t *= 10.0 / m0
        rcl = cutoff(t)
    cs = cs_of(rcl, t)
    ms = [good_size(math.ceil(cs * L / (math.pi * rcl * Lmin)), mult) for L in Lv]
    hs = [float(L) / m for L, m in zip(Lv, ms)]
    hmax = max(hs)
    rcl = cs * hmax / (math.pi * Lmin)
    cw = cw_of(cs_of(rcl, t_pot), rcl)      # window balanced against the potential target
    P = int(math.ceil(2.0 * (rcl * cw / cs) * Lmin / hmax))
    return dict(L=[float(L) for L in Lv], rc=rcl * Lmin, cs=cs, cw_target=cw, cw=math.pi * P / 2.0, m=ms, P=P,
                h=hs, alpha=[P * h / 2.0 for h in hs])
