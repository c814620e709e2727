"""Alg. 2 (fast Fourier-space sum) restated step by step, plain FP64 (oracle; test use only).

Given the plan's (m, P, cs, cw, rc) for a box [0, L)^3, with h = L/m and the
window half-width alpha = P h / 2 (Sec. 6.3, eq. alpha and the relation alpha = P L/(2m)):

1. spread   a_l = sum_j rho_j phitilde(x_j - h l)                       (Alg. 2 step 1, eq. spread_def)
            phi^{cw}(y) = prod_i psi^{cw}(y_i/alpha)/psi^{cw}(0) on [-alpha, alpha]^3
            Each particle touches the P grid points l0..l0+P-1 per axis,
            l0 = ceil(x/h - P/2) (the points with x - h l in (-alpha, alpha]);
            indices are taken mod m (periodisation).
2. FFT      ahat_k = sum_l a_l e^{+2 pi i k.l/m}                          (Alg. 2 step 2)
3. scale    bhat_k = S(k) ahat_k,  S(0) = 0,
            S(k) = (1/V) Mhat(k) / [phihat(k)/h^3]^2                      (Alg. 2 step 3, eq. diag_scale)
            phihat(k)/h^3 = prod_i (1/h) int phi_1d(y) e^{-i w_i y} dy,  w_i = 2 pi k_i/L.
            The factor h^-3 converts the continuous transform of Sec. 4.3 into the
            coefficient seen by an unnormalised m^3-point DFT (Poisson summation with
            c_k = phihat/V of eq. fcoeffs, times m^3); Alg. 2 as printed leaves it implicit.
            Retained modes: k in I_m strictly inside the mollifier's band,
            |w| < c_s/r_c (eq. csrc; |k| < c_s L/(2 pi r_c) for a cube), with the unpaired
            Nyquist planes k_d = -m_d/2 of an even m_d dropped.  Prop. 1 bounds the split
            error by the modes outside this band, and deconvolving where phihat ~ psi(1)^3
            (cube corners) or at an aliased Nyquist plane amplifies rounding by up to
            ~exp(3 c_w - c_s).  When eq. csrc holds exactly (instantiated plans) the band is
            the open ball |k| < m/2.  ``modes="cube"`` keeps the whole cube I_m of Alg. 2 as
            printed, for comparison.
4. IFFT     b_l = sum_k bhat_k e^{-2 pi i k.l/m}                          (Alg. 2 step 4)
5. interp   phi_i^far = sum_l b_l phitilde(x_i - h l)                     (Alg. 2 step 5)
            grad phi_i^far = sum_l b_l grad phitilde(x_i - h l)           (Remark 'force', eq. force)
            d/dy_j phi = (1/alpha) psi'(y_j/alpha) prod_{i != j} psi(y_i/alpha) / psi(0)^3

psi is evaluated exactly from its Legendre series (no polynomial fits), the
FFTs are NumPy's complex FFTs, and k runs over I_m = {-m/2, ..., m/2-1}.

Cuboid boxes (Remark on cuboid domains, Sec. 6.1): L and m may be given per axis; then h_d = L_d/m_d,
alpha_d = P h_d/2 (the window support is P points on every axis), w_d = 2 pi k_d/L_d, V = prod L_d,
and the band |w| < c_s/r_c is the ellipsoid 0 < |w| < pi min_d m_d/L_d once r_c is
instantiated from the coarsest axis (eq. csrc).

Parity status: pinned (tests/test_oracle_alg2.py) against the converged Ewald sum
of ``exact`` (its difference is the method's own error, compared with the error
models of Sec. 5), by a single-charge DFT identity, and (tests/test_oracle_table3.py)
by the paper's Table 3: the smallest (m, P) that reach each tolerance in its n = 100,
r_c = 0.1, c_s = log(1/eps) experiment.
"""
import numpy as np

from .pswf import PSWF
from .split import PSWFSplit
from .exact import wrap, realspace


class Alg2:
    def __init__(self, L, m, P, cs, cw, rc, modes="band"):
        if modes not in ("band", "cube"):
            raise ValueError("modes must be 'band' or 'cube'")
        self.modes = modes
        self.Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
        self.mv = np.broadcast_to(np.asarray(m, dtype=np.int64), (3,)).copy()
        self.P = int(P)
        self.cs, self.cw, self.rc = float(cs), float(cw), float(rc)
        self.hv = self.Lv / self.mv
        self.alphav = self.P * self.hv / 2.0
        # scalar views (cubes)
        self.L, self.m, self.h, self.alpha = float(self.Lv[0]), int(self.mv[0]), float(self.hv[0]), float(self.alphav[0])
        self.win = PSWF(self.cw)
        self.split = PSWFSplit(self.cs, self.rc)

    # -- window ------------------------------------------------------------------
    def _stencil(self, x):
        """Per-axis grid indices (n,3,P) and window arguments s = (x - h l)/alpha."""
        h, al, mv = self.hv[None, :, None], self.alphav[None, :, None], self.mv[None, :, None]
        t = x / self.hv[None, :]
        l0 = np.ceil(t - self.P / 2.0)
        a = np.arange(self.P, dtype=np.float64)
        l = l0[:, :, None] + a[None, None, :]
        s = (x[:, :, None] - h * l) / al
        idx = np.mod(l.astype(np.int64), mv)
        return idx, s

    def window_1d(self, s):
        return self.win.psi(s) / self.win.psi0

    def dwindow_1d(self, s):
        """d/dy of the window on every axis (s has the axis as its second index)."""
        return self.win.dpsi(s) / (self.win.psi0 * self.alphav[None, :, None])

    # -- Alg. 2 steps -----------------------------------------------------------
    def spread(self, x, rho, chunk=4096):
        x = wrap(x, self.Lv)
        (mx, my, mz), P = self.mv, self.P
        a = np.zeros(mx * my * mz)
        for s0 in range(0, len(x), chunk):
            idx, s = self._stencil(x[s0:s0 + chunk])
            w = self.window_1d(s)
            r = np.asarray(rho[s0:s0 + chunk], dtype=np.float64)
            vals = (r[:, None, None, None] * w[:, 0, :, None, None]
                    * w[:, 1, None, :, None] * w[:, 2, None, None, :])
            flat = (idx[:, 0, :, None, None] * my + idx[:, 1, None, :, None]) * mz + idx[:, 2, None, None, :]
            a += np.bincount(flat.ravel(), weights=vals.ravel(), minlength=mx * my * mz)
        return a.reshape(mx, my, mz)

    def kgrid(self, axis=0):
        """Integer k in I_m for each FFT index of an axis (index m/2 is k = -m/2)."""
        m = int(self.mv[axis])
        return np.rint(np.fft.fftfreq(m) * m).astype(np.int64)

    def window_ft(self, axis):
        """(1/h) int_{-alpha}^{alpha} psi(y/alpha)/psi(0) cos(w y) dy for the FFT indices of an axis."""
        w = 2.0 * np.pi * self.kgrid(axis) / self.Lv[axis]
        al = self.alphav[axis]
        return al * self.win.cos_transform(w * al) / (self.win.psi0 * self.hv[axis])

    def scaling(self):
        """S(k) on the full index grid (S(0) = 0; zero outside the retained modes)."""
        ph = [self.window_ft(d) for d in range(3)]
        den = (ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]) ** 2
        ks = [self.kgrid(d) for d in range(3)]
        KX, KY, KZ = np.meshgrid(*ks, indexing='ij')
        cube = np.all(self.Lv == self.Lv[0]) and np.all(self.mv == self.mv[0])
        S = np.zeros(KX.shape)
        if cube:
            L = self.L
            k2 = KX ** 2 + KY ** 2 + KZ ** 2
            nz = k2 > 0
            uk, inv = np.unique(k2[nz], return_inverse=True)
            S[nz] = self.split.Mhat_k2(uk, L)[inv] / (L ** 3) / den[nz]
            w2 = (2.0 * np.pi / L) ** 2 * k2
        else:
            w2 = (2.0 * np.pi) ** 2 * ((KX / self.Lv[0]) ** 2 + (KY / self.Lv[1]) ** 2 + (KZ / self.Lv[2]) ** 2)
            nz = w2 > 0
            uw, inv = np.unique(w2[nz], return_inverse=True)
            S[nz] = self.split.Mhat_w2(uw)[inv] / float(np.prod(self.Lv)) / den[nz]
        if self.modes == "band":
            wb = self.cs / self.rc                       # eq. csrc: the mollifier's bandlimit
            S[w2 >= wb * wb * (1.0 - 1e-12)] = 0.0       # (a band edge at exactly m/2 counts as outside)
            for d, K in enumerate((KX, KY, KZ)):
                if self.mv[d] % 2 == 0:
                    S[K == -(self.mv[d] // 2)] = 0.0
        return S

    def fft(self, a):
        return np.fft.ifftn(a) * a.size                  # e^{+2 pi i k.l/m}, unnormalised

    def ifft(self, bh):
        return np.fft.fftn(bh)                           # e^{-2 pi i k.l/m}, unnormalised

    def interp(self, x, b, chunk=4096):
        x = wrap(x, self.Lv)
        mx, my, mz = self.mv
        bf = b.ravel()
        phi = np.zeros(len(x))
        grad = np.zeros((len(x), 3))
        for s0 in range(0, len(x), chunk):
            idx, s = self._stencil(x[s0:s0 + chunk])
            w = self.window_1d(s)
            dw = self.dwindow_1d(s)
            flat = (idx[:, 0, :, None, None] * my + idx[:, 1, None, :, None]) * mz + idx[:, 2, None, None, :]
            G = bf[flat]                                  # (c, P, P, P)
            # contract the z axis, then y, then x (plain tensor contractions)
            Gz = np.einsum('nabc,nc->nab', G, w[:, 2])
            Gdz = np.einsum('nabc,nc->nab', G, dw[:, 2])
            Gzy = np.einsum('nab,nb->na', Gz, w[:, 1])
            Gzdy = np.einsum('nab,nb->na', Gz, dw[:, 1])
            Gdzy = np.einsum('nab,nb->na', Gdz, w[:, 1])
            sl = slice(s0, s0 + chunk)
            phi[sl] = np.einsum('na,na->n', Gzy, w[:, 0])
            grad[sl, 0] = np.einsum('na,na->n', Gzy, dw[:, 0])
            grad[sl, 1] = np.einsum('na,na->n', Gzdy, w[:, 0])
            grad[sl, 2] = np.einsum('na,na->n', Gdzy, w[:, 0])
        return phi, grad

    def far(self, x, rho, stages=False, targets=None):
        a = self.spread(x, rho)
        ah = self.fft(a)
        bh = self.scaling() * ah
        b = np.real(self.ifft(bh))
        xt = x if targets is None else np.asarray(x)[targets]
        phi, grad = self.interp(xt, b)
        if stages:
            return phi, grad, {"a": a, "ahat": ah, "bhat": bh, "b": b}
        return phi, grad

    def total(self, x, rho, stages=False, targets=None):
        """phi, grad phi, E, F of the fast method (far + local + self) on CPU."""
        rho = np.asarray(rho, dtype=np.float64)
        out = self.far(x, rho, stages=stages, targets=targets)
        pf, gf = out[0], out[1]
        pl, gl = realspace(x, rho, self.Lv, self.split, self.rc, targets=targets)
        if targets is not None:
            r = rho[targets]
        else:
            r = rho
        phi = pl + pf - self.split.self_coeff() * r
        grad = gl + gf
        F = -r[:, None] * grad
        E = 0.5 * float(np.dot(rho, phi)) if targets is None else None
        if stages:
            return phi, grad, E, F, out[2]
        return phi, grad, E, F
