"""Alg. 3 parameter selection (Sec. 6), plain FP64 with scipy's Lambert W (oracle; test use only).

This module holds the paper's procedure and nothing else.  The CUDA library's planner adds
rules of its own on top of it (how it picks r_c, the rounding of m, a tighter target for the
split and the safety factor); the planner tests state those as explicit differences from
this procedure instead of restating them here.

Alg. 3 takes a tolerance eps and a cutoff r_c (the paper leaves r_c to runtime tuning,
Sec. 6.2.2) and returns (c_s, c_w, alpha, m, P):

1. c_s = W_0(2 (B_s/eps)^2)/2,  B_s = A_s ||rho||_2 sqrt(r_c)/sqrt(V)    (eq. cs_dimless)
2. c_w = -W_{-1}(-2 B_w^2 e^{-2 c_s}/c_s)/2,  B_w = (A_s/A_w) sqrt(r_c/L)   (eq. cwW)
3. alpha = r_c c_w / c_s                                                  (eq. alpha)
4. m = ceil(L c_s/(pi r_c))                                               (eq. m_cs_dimless)
5. P = ceil(2 alpha m / L)                                                (eq. P_dimless)

Readings (the paper is silent on them):

* Relative tolerance.  Alg. 3 targets an absolute RMS error eps.  A relative tolerance tol
  maps to eps = tol sqrt(kappa) ||rho||_2 / L, where kappa = pi^-2 sum_{k != 0} |k|^-4 is the
  mean square of the neutralised periodic potential of unit-norm uniform charges (Parseval
  with c_k = Mhat/V, eq. fcoeffs).  Then B_s/eps = A_s sqrt(r_c/L) / (sqrt(kappa) tol)
  needs no rho.
* Lambert-W branches: W_0 for c_s (its argument is positive), W_{-1} for c_w (the argument
  lies in (-1/e, 0); the large root is the meaningful one).
* Instantiation after rounding.  Alg. 2 needs eq. csrc (c_s/r_c = pi m/L) and eq. bandwidth
  (c_s/r_c = c_w/alpha) to hold exactly once m and P are integers.  ``instantiate`` keeps c_s,
  sets r_c := c_s L/(pi m) (the split error can only drop), c_w := pi P/2 and alpha := P h/2
  (eq. cwP), so the window transform arguments 2 k_i/m stay in [-1, 1].

Parity: pinned in tests/test_oracle_alg2.py by Lambert-W identities, by the balance
equation eq. cwcs_model_dimless that eq. cwW solves, by kappa against a direct lattice sum,
by the exact relations of steps 3-5 and eq. cwP after instantiation, by the ratio A_s/A_w the
paper states (Sec. 6.3), and by the measured potential error of Alg. 2 with these parameters
(close to tol, as the Remark after Alg. 3 states); Table 3's smallest (m, P) are reproduced
through the Alg. 2 oracle in tests/test_oracle_table3.py.
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


def bs_over_eps(rc_over_L, tol):
    """B_s/eps of eq. cs_dimless under the relative-tolerance reading (no rho needed)."""
    return A_S * math.sqrt(rc_over_L) / (math.sqrt(KAPPA) * tol)


def cs_of(rc_over_L, tol):
    """Alg. 3 step 1 (eq. cs_dimless), principal branch."""
    return 0.5 * float(np.real(lambertw(2.0 * bs_over_eps(rc_over_L, tol) ** 2, 0)))


def cw_of(cs, rc_over_L):
    """Alg. 3 step 2 (eq. cwW), lower branch."""
    bw = (A_S / A_W) * math.sqrt(rc_over_L)
    z = -2.0 * bw * bw * math.exp(-2.0 * cs) / cs
    return -0.5 * float(np.real(lambertw(z, -1)))


def alg3(L, tol, rc, cs=None):
    """Alg. 3 steps 1-5 for a cube of edge L: dict(cs, cw, alpha, m, P).

    ``cs`` overrides step 1 (the paper's alternative c_s = log(1/eps), used by Table 3).
    """
    rcl = rc / L
    if cs is None:
        cs = cs_of(rcl, tol)
    cw = cw_of(cs, rcl)
    alpha = rc * cw / cs
    m = int(math.ceil(L * cs / (math.pi * rc)))
    P = int(math.ceil(2.0 * alpha * m / L))
    return dict(cs=cs, cw=cw, alpha=alpha, m=m, P=P)


def instantiate(L, m, P, cs):
    """Effective parameters for Alg. 2 after rounding (reading above): eq. csrc and eq. cwP exact."""
    h = L / m
    return dict(L=L, m=m, P=P, cs=cs, rc=cs * L / (math.pi * m), cw=math.pi * P / 2.0, h=h, alpha=P * h / 2.0)


def split_model(cs, rc_over_L):
    """Right-hand side of eq. cwcs_model_dimless (L = 1 units): sqrt(rc) A_s c_s^-1/2 e^-c_s."""
    return math.sqrt(rc_over_L) * A_S * cs ** -0.5 * math.exp(-cs)


def window_model(cw):
    """Left-hand side of eq. cwcs_model_dimless (L = 1 units): A_w c_w^1/2 e^-c_w."""
    return A_W * math.sqrt(cw) * math.exp(-cw)


def even_up(m):
    """The paper assumes an even m (Sec. 6.3, before eq. cwP)."""
    m = int(m)
    return m + (m % 2)


def plan(L, tol, rc, cs=None):
    """Alg. 3 for a cube at cutoff rc, m rounded up to even, then instantiated (reading above)."""
    q = alg3(L, tol, rc, cs=cs)
    m = even_up(q["m"])
    P = int(math.ceil(2.0 * q["alpha"] * m / L))
    out = instantiate(L, m, P, q["cs"])
    out["cw_target"] = q["cw"]
    return out


def plan_box(Ls, tol, rc):
    """Alg. 3 for a cuboid box (Remark on cuboid domains, Sec. 6.1, which gives no parameter rule).

    Reading: the procedure runs in units of the shortest edge L_min (r_c/L_min in steps 1-2);
    every axis gets m_d = ceil(c_s L_d/(pi r_c)), made even; then r_c := c_s h_max/pi (eq. csrc on
    the coarsest axis) and P = ceil(2 alpha/h_max) with alpha = r_c c_w/c_s, instantiated as
    c_w := pi P/2 and alpha_d := P h_d/2.  Equal edges give ``plan``.
    """
    Lv = np.broadcast_to(np.asarray(Ls, dtype=np.float64), (3,))
    if np.all(Lv == Lv[0]):
        q = plan(float(Lv[0]), tol, rc)
        q.update(m=[q["m"]] * 3, h=[q["h"]] * 3, alpha=[q["alpha"]] * 3, L=[q["L"]] * 3)
        return q
    Lmin = float(np.min(Lv))
    rcl = rc / Lmin
    cs = cs_of(rcl, tol)
    ms = [even_up(math.ceil(cs * float(L) / (math.pi * rc))) for L in Lv]
    hs = [float(L) / m for L, m in zip(Lv, ms)]
    hmax = max(hs)
    rcn = cs * hmax / math.pi
    cw = cw_of(cs, rcn / Lmin)
    P = int(math.ceil(2.0 * (rcn * cw / cs) / hmax))
    return dict(L=[float(L) for L in Lv], rc=rcn, cs=cs, cw_target=cw, cw=math.pi * P / 2.0, m=ms, P=P,
                h=hs, alpha=[P * h / 2.0 for h in hs])
