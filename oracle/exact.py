"""Converged triply periodic Ewald sums, plain FP64 (oracle; test use only).

The potential at x_i (Sec. 3.1, eqs. potential2 / Ewald decomposition):
  phi_i = phi_i^local + phi_i^far + phi_i^self
  phi_i^local = sum_{r in Z^3} sum_j' rho_j R(|x_i - x_j + L r|)          (real space)
  phi_i^far   = (1/V) sum_{k != 0} Mhat(k) Re[rhohat(k) e^{-2 pi i k.x_i/L}],
                rhohat(k) = sum_j rho_j e^{+2 pi i k.x_j/L}                 (Alg. 1, eq. Fsum)
  phi_i^self  = -lim_{r->0} M(r) rho_i
  E = 1/2 sum_i rho_i phi_i,   F_i = -rho_i grad phi_i                    (Remark after eq. Ewald)
The k-sum runs over the whole sphere |k| <= K (not truncated to I_m); the
caller picks K so that the omitted tail is below the test tolerance.  The prime
omits (j = i, r = 0).

``lattice_shell_sum`` is the brute-force replica sum of 1/r over cubic shells
|r|_inf <= N, used to pin the Ewald result on tiny neutral systems.

Boxes may be cuboids (Remark on cuboid domains in Sec. 6.1): ``L`` is a scalar
edge or the three edges (L_x, L_y, L_z); images are x + (r_x L_x, r_y L_y, r_z L_z),
wave vectors omega = 2 pi (k_x/L_x, k_y/L_y, k_z/L_z), V = L_x L_y L_z, and the
Fourier sum runs over the ellipsoid |omega| <= omega_max.

Parity status: pinned (tests/test_oracle_exact.py) by split independence
(two PSWF cutoffs and the Gaussian split agree), the NaCl Madelung constant,
brute-force lattice sums, translation invariance, the scaling law of
eq. phinondim and sum_i F_i = 0.
"""
import numpy as np


def box(L):
    """The three box edges as an array (a scalar L is a cube)."""
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    return Lv


def wrap(x, L):
    """Map positions into the periodic box prod_i [0, L_i)."""
    Lv = box(L)
    x = np.mod(np.asarray(x, dtype=np.float64), Lv)
    return np.where(x >= Lv, x - Lv, x)


def realspace(x, rho, L, split, rcut, targets=None, chunk=64):
    """phi^local and grad phi^local at the targets (all particles by default).

    Sums every periodic image within ``rcut`` of the target.
    """
    Lv = box(L)
    x = wrap(x, Lv)
    rho = np.asarray(rho, dtype=np.float64)
    tgt = np.arange(len(x)) if targets is None else np.asarray(targets)
    if rcut <= 0.5 * np.min(Lv):
        # any image other than the minimum one is at least min(L)/2 away
        shifts = np.zeros((1, 3))
    else:
        rngs = [np.arange(-int(np.ceil(rcut / Li)), int(np.ceil(rcut / Li)) + 1) for Li in Lv]
        shifts = np.array([(a, b, c) for a in rngs[0] for b in rngs[1] for c in rngs[2]], dtype=np.float64) * Lv
    phi = np.zeros(len(tgt))
    grad = np.zeros((len(tgt), 3))
    chunk = max(1, min(chunk, (1 << 24) // max(len(x), 1)))   # memory only: ~0.4 GB per (t, n, 3) array
    for s in range(0, len(tgt), chunk):
        ti = tgt[s:s + chunk]
        d0 = x[ti, None, :] - x[None, :, :]
        d0 -= Lv * np.round(d0 / Lv)             # minimum image, then explicit shells
        for sh in shifts:
            d = d0 + sh
            r = np.sqrt(np.sum(d * d, axis=-1))
            mask = (r < rcut) & (r > 0.0)                # r = 0 only for the omitted self pair
            tt, jj = np.nonzero(mask)
            if len(tt) == 0:
                continue
            rr = r[tt, jj]
            Rv, dRv = split.R_and_dR(rr)
            phi[s:s + chunk] += np.bincount(tt, weights=Rv * rho[jj], minlength=len(ti))
            coef = dRv / rr * rho[jj]
            for dim in range(3):
                grad[s:s + chunk, dim] += np.bincount(tt, weights=coef * d[tt, jj, dim], minlength=len(ti))
    return phi, grad


def structure_factor(x, rho, L, K, chunk=250_000):
    """rhohat(k) = sum_j rho_j exp(+2 pi i sum_d k_d x_jd / L_d) on the box |k_d| <= K_d.

    K is an integer (all axes) or three integers.  The sum over j is accumulated over blocks of
    particles (memory only)."""
    Lv = box(L)
    Kv = np.broadcast_to(np.asarray(K, dtype=np.int64), (3,))
    x = wrap(x, Lv)
    rho = np.asarray(rho, dtype=np.float64)
    kr = [np.arange(-k, k + 1) for k in Kv]
    rh = np.zeros(tuple(2 * k + 1 for k in Kv), dtype=np.complex128)
    for s0 in range(0, len(x), chunk):
        xs, rs = x[s0:s0 + chunk], rho[s0:s0 + chunk]
        Ex, Ey, Ez = (np.exp(2j * np.pi * xs[:, d, None] * kr[d][None, :] / Lv[d]) for d in range(3))
        for ix in range(2 * Kv[0] + 1):
            A = (rs * Ex[:, ix])[:, None] * Ey
            rh[ix] += A.T @ Ez
    return rh


def kspace(x, rho, L, split, K, targets=None):
    """phi^far and grad phi^far from the direct Fourier sum over 0 < |omega| <= omega_max.

    Cube (scalar L and K): the sphere 0 < |k| <= K.  Cuboid: K = (K_x, K_y, K_z) and the ellipsoid
    |omega| <= omega_max = 2 pi min_d K_d / L_d, omega_d = 2 pi k_d / L_d."""
    Lv = box(L)
    Kv = np.broadcast_to(np.asarray(K, dtype=np.int64), (3,))
    x = wrap(x, Lv)
    V = float(np.prod(Lv))
    kr = [np.arange(-k, k + 1) for k in Kv]
    KX, KY, KZ = np.meshgrid(*kr, indexing='ij')
    if np.all(Lv == Lv[0]) and np.all(Kv == Kv[0]):
        k2 = KX ** 2 + KY ** 2 + KZ ** 2
        mask = (k2 > 0) & (k2 <= Kv[0] * Kv[0])
        Mh = np.zeros(k2.shape)
        uk, inv = np.unique(k2[mask], return_inverse=True)
        Mh[mask] = split.Mhat_k2(uk.astype(np.float64), Lv[0])[inv]
    else:
        w2 = (2.0 * np.pi) ** 2 * ((KX / Lv[0]) ** 2 + (KY / Lv[1]) ** 2 + (KZ / Lv[2]) ** 2)
        wmax = 2.0 * np.pi * np.min(Kv / Lv)
        mask = (w2 > 0) & (w2 <= wmax * wmax)
        Mh = np.zeros(w2.shape)
        uw, inv = np.unique(w2[mask], return_inverse=True)
        Mh[mask] = split.Mhat_w2(uw)[inv]
    C = Mh * structure_factor(x, rho, Lv, Kv) / V        # (1/V) Mhat rhohat
    tgt = np.arange(len(x)) if targets is None else np.asarray(targets)
    xt = x[tgt]
    Ex, Ey, Ez = (np.exp(-2j * np.pi * xt[:, d, None] * kr[d][None, :] / Lv[d]) for d in range(3))
    fac = [-2j * np.pi * kr[d] / Lv[d] for d in range(3)]
    phi = np.zeros(len(tgt))
    grad = np.zeros((len(tgt), 3))
    for ix in range(2 * Kv[0] + 1):
        B = Ex[:, ix][:, None] * Ey                     # (t, ky)
        T = B @ C[ix]                                   # (t, kz): sum over ky
        Ty = (B * fac[1][None, :]) @ C[ix]
        phi += np.real(np.sum(T * Ez, axis=1))
        grad[:, 0] += np.real(fac[0][ix] * np.sum(T * Ez, axis=1))
        grad[:, 1] += np.real(np.sum(Ty * Ez, axis=1))
        grad[:, 2] += np.real(np.sum(T * Ez * fac[2][None, :], axis=1))
    return phi, grad


def ewald(x, rho, L, split, K, rcut, targets=None):
    """Total phi, grad phi, energy (only when all particles are targets) and forces."""
    rho = np.asarray(rho, dtype=np.float64)
    pl, gl = realspace(x, rho, L, split, rcut, targets)
    pf, gf = kspace(x, rho, L, split, K, targets)
    tgt = np.arange(len(rho)) if targets is None else np.asarray(targets)
    phi = pl + pf - split.self_coeff() * rho[tgt]
    grad = gl + gf
    F = -rho[tgt, None] * grad
    E = 0.5 * float(np.dot(rho, phi)) if targets is None else None
    return phi, grad, E, F


def pswf_exact(x, rho, L, cs=34.0, rc_frac=0.5, kfac=1.25, targets=None):
    """O-exact with the oracle's own PSWF split (cs ~ 34, rc = rc_frac min(L))."""
    from .split import PSWFSplit
    Lv = box(L)
    rc = rc_frac * float(np.min(Lv))
    K = [int(np.ceil(kfac * cs * Li / (2.0 * np.pi * rc))) for Li in Lv]
    if np.all(Lv == Lv[0]):
        return ewald(x, rho, Lv[0], PSWFSplit(cs, rc), K[0], rc, targets)
    return ewald(x, rho, Lv, PSWFSplit(cs, rc), K, rc, targets)


def gaussian_exact(x, rho, L, xi=6.0, targets=None):
    """Classical erfc Ewald: real space cut at min(L)/2, sigma = min(L)/(2 xi), k-range to e^{-...} < 1e-17."""
    from .split import GaussianSplit
    Lv = box(L)
    sigma = float(np.min(Lv)) / (2.0 * xi)
    # exp(-sigma^2 w^2 / 4) < 1e-17  <=>  w > 2 sqrt(17 ln 10)/sigma
    wmax = 2.0 * np.sqrt(17.0 * np.log(10.0)) / sigma
    K = [int(np.ceil(wmax * Li / (2.0 * np.pi))) for Li in Lv]
    if np.all(Lv == Lv[0]):
        return ewald(x, rho, Lv[0], GaussianSplit(sigma), K[0], 0.5 * Lv[0], targets)
    return ewald(x, rho, Lv, GaussianSplit(sigma), K, 0.5 * float(np.min(Lv)), targets)


def lattice_shell_sum(x, rho, L, N):
    """Brute force: phi_i and grad phi_i summed over whole replicas |r|_inf <= N (self excluded)."""
    x = np.asarray(x, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    n = len(x)
    rng = np.arange(-N, N + 1, dtype=np.float64)
    R = np.stack(np.meshgrid(rng, rng, rng, indexing='ij'), axis=-1).reshape(-1, 3) * L
    phi = np.zeros(n)
    grad = np.zeros((n, 3))
    for i in range(n):
        for j in range(n):
            d = x[i] - x[j] + R                      # (nimg, 3)
            r2 = np.sum(d * d, axis=1)
            if i == j:
                r2 = np.where(r2 == 0.0, np.inf, r2)
            r = np.sqrt(r2)
            phi[i] += rho[j] * np.sum(1.0 / r)
            grad[i] -= rho[j] * np.sum(d / (r ** 3)[:, None], axis=0)
    return phi, grad
