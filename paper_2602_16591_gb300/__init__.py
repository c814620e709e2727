"""GB300 PSWF fast Ewald summation: thin Python binding over libpswf_ewald.so.

Every step of the evaluation runs in the library's CUDA kernels (and cuFFT);
this module only marshals arguments (ctypes) and uses PyTorch for device
memory and streams.  There is no CPU fallback: importing the package fails
loudly when the shared library has not been built (``python -m
paper_2602_16591_gb300.build``).

The names follow the C ABI in ``include/pswf_ewald.h``.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpswf_ewald.so")

EWALD_OK, EWALD_EINVAL, EWALD_ENONNEUTRAL, EWALD_ENOMEM = 0, 1, 2, 3
EWALD_ECUDA, EWALD_ECUFFT, EWALD_ETOOBIG, EWALD_ETIMEOUT, EWALD_ENONFINITE = 4, 5, 6, 7, 8
EWALD_FP64, EWALD_MIXED, EWALD_FLOATFLOAT = 0, 1, 2
PRECISIONS = {"fp64": EWALD_FP64, "mixed": EWALD_MIXED, "floatfloat": EWALD_FLOATFLOAT}
PATH_NAMES = {EWALD_FP64: "f64", EWALD_MIXED: "f32", EWALD_FLOATFLOAT: "ff"}


class ewald_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rc", ctypes.c_double), ("grid_density", ctypes.c_double),
                ("tol_safety", ctypes.c_double), ("sr_reach", ctypes.c_int), ("window_extra", ctypes.c_int),
                ("autotune", ctypes.c_int), ("spread_kernel", ctypes.c_int)]


class ewald_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("L", "rc", "cs", "cw", "cw_target", "alpha", "h", "lambda_s", "lambda_w", "self_coeff",
                 "tol", "fit_tol")] + [("n", ctypes.c_int64)] + [(k, ctypes.c_int) for k in
                ("m", "P", "deg_w", "deg_r", "tile", "ncell", "sr_reach", "precision")] + \
        [("box", ctypes.c_double * 3), ("grid", ctypes.c_int * 3), ("cells", ctypes.c_int * 3), ("deg_g", ctypes.c_int),
         ("sr_reach_z", ctypes.c_int), ("spread_kernel", ctypes.c_int)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k in ("box", "grid", "cells") else v
        return out


class EwaldError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d): %s" % (_lib.ewald_error_string(code).decode(), code, msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpswf_ewald.so is not built; run `python paper_2602_16591_gb300/build.py` "
                          "(nvcc, sm_103a) -- there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "ewald_opts_default": (I, [ctypes.POINTER(ewald_opts)]),
        "ewald_plan_params": (I, [D, I64, D, ctypes.POINTER(ewald_opts), ctypes.POINTER(ewald_params)]),
        "ewald_plan_create": (I, [D, I64, D, ctypes.POINTER(ewald_opts), ctypes.POINTER(P)]),
        "ewald_plan_params_box": (I, [P, I64, D, ctypes.POINTER(ewald_opts), ctypes.POINTER(ewald_params)]),
        "ewald_plan_create_box": (I, [P, I64, D, ctypes.POINTER(ewald_opts), ctypes.POINTER(P)]),
        "ewald_plan_query": (I, [P, ctypes.POINTER(ewald_params)]),
        "ewald_eval": (I, [P, P, P, P, P, dp, P]),
        "ewald_eval_host": (I, [P, P, P, P, P, dp, P]),
        "ewald_check": (I, [P, P]),
        "ewald_debug_grid": (I, [P, I, P]),
        "ewald_plan_destroy": (None, [P]),
        "ewald_pswf_eval": (I, [D, I, P, P, P, dp, dp]),
        "ewald_lambertw": (D, [I, D]),
        "ewald_window_fit": (I, [ctypes.POINTER(ewald_params), I, P, P, P]),
        "ewald_radial_fit": (I, [ctypes.POINTER(ewald_params), I, P, P, P]),
        "ewald_scale_table": (I, [ctypes.POINTER(ewald_params), P]),
        "ewald_profile": (I, [P, I]),
        "ewald_profile_read": (I, [P, P, ctypes.POINTER(ctypes.c_int)]),
        "ewald_debug_wait_timeout": (I, []),
        "ewald_spread_static": (I, [ctypes.POINTER(ewald_params), P, P, P, P]),
        "ewald_plan_batch_create": (I, [I, P, P, D, ctypes.POINTER(ewald_opts), ctypes.POINTER(P)]),
        "ewald_eval_batch": (I, [P, P, P, P, P, P, P, P]),
        "ewald_error_string": (ctypes.c_char_p, [I]),
        "ewald_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
lib = _lib


def _check(code):
    if code != EWALD_OK:
        raise EwaldError(code, _lib.ewald_last_error().decode())


def make_opts(precision="fp64", rc=None, grid_density=None, tol_safety=None, sr_reach=None, window_extra=None,
              autotune=None, spread_kernel=None):
    o = ewald_opts()
    _check(_lib.ewald_opts_default(ctypes.byref(o)))
    if isinstance(precision, str):
        if precision not in PRECISIONS:
            raise ValueError("precision must be one of %s" % ", ".join(sorted(PRECISIONS)))
        o.precision = PRECISIONS[precision]
    else:
        o.precision = int(precision)
    if rc is not None:
        o.rc = float(rc)
    if grid_density is not None:
        o.grid_density = float(grid_density)
    if tol_safety is not None:
        o.tol_safety = float(tol_safety)
    if sr_reach is not None:
        o.sr_reach = int(sr_reach)
    if window_extra is not None:
        o.window_extra = int(window_extra)
    if autotune is not None:
        o.autotune = int(bool(autotune))
    if spread_kernel is not None:
        o.spread_kernel = int(spread_kernel)
    return o


def _box(L):
    """(L, is_cube): a scalar edge or three edges (cuboid box) as a C double[3]."""
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    return (ctypes.c_double * 3)(*[float(v) for v in Lv]), bool(np.ndim(L) == 0)


def plan_params(L, n, tol, **opts):
    """Alg. 3 parameters on the host (no GPU needed).  L: edge of a cube, or three edges of a cuboid."""
    o = make_opts(**opts)
    p = ewald_params()
    box, cube = _box(L)
    if cube:
        _check(_lib.ewald_plan_params(float(L), int(n), float(tol), ctypes.byref(o), ctypes.byref(p)))
    else:
        _check(_lib.ewald_plan_params_box(box, int(n), float(tol), ctypes.byref(o), ctypes.byref(p)))
    return p


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _out(a, shape):
    """A caller's float64 output array (written in place), or a new one when a is None."""
    if a is None:
        return np.empty(shape)
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or a.shape != shape \
            or not a.flags.c_contiguous or not a.flags.writeable:
        raise ValueError("output must be a writeable C-contiguous float64 array of shape %s" % (shape,))
    return a


def pswf_eval(c, x):
    """The library planner's psi_0^c, its derivative, chi_0 and lambda_0 (host)."""
    x = _f64(x).ravel()
    psi = np.empty_like(x)
    dpsi = np.empty_like(x)
    chi = ctypes.c_double()
    lam = ctypes.c_double()
    _check(_lib.ewald_pswf_eval(float(c), len(x), _ptr(x), _ptr(psi), _ptr(dpsi), ctypes.byref(chi), ctypes.byref(lam)))
    return psi, dpsi, chi.value, lam.value


def lambertw(branch, z):
    return _lib.ewald_lambertw(int(branch), float(z))


def window_fit(params, z):
    z = _f64(z).ravel()
    w = np.empty((len(z), params.P))
    dw = np.empty((len(z), params.P))
    _check(_lib.ewald_window_fit(ctypes.byref(params), len(z), _ptr(z), _ptr(w), _ptr(dw)))
    return w, dw


def radial_fit(params, r):
    r = _f64(r).ravel()
    R = np.empty_like(r)
    G = np.empty_like(r)
    _check(_lib.ewald_radial_fit(ctypes.byref(params), len(r), _ptr(r), _ptr(R), _ptr(G)))
    return R, G


def scale_table(params):
    mx, my, mz = (int(v) for v in params.grid)
    S = np.empty((mx, my, mz // 2 + 1))
    _check(_lib.ewald_scale_table(ctypes.byref(params), _ptr(S)))
    return S


class Plan:
    """A PSWF Ewald plan on the current CUDA device (C ABI: ewald_plan_create).

    ``L`` is the edge of a cube or the three edges of a cuboid box.  ``precision`` is "fp64", "mixed" or "floatfloat" ("mixed" below tol 1e-7 runs the float-float
    kernels; ``params.precision`` reports the path); other keywords are the ewald_opts fields.
    """

    def __init__(self, L, n, tol, precision="fp64", **opts):
        import torch  # device memory and streams only
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("PSWF Ewald plans need a CUDA device (no CPU fallback)")
        torch.cuda.init()
        self.device = torch.device("cuda", torch.cuda.current_device())
        o = make_opts(precision=precision, **opts)
        h = ctypes.c_void_p()
        box, cube = _box(L)
        if cube:
            _check(_lib.ewald_plan_create(float(L), int(n), float(tol), ctypes.byref(o), ctypes.byref(h)))
        else:
            _check(_lib.ewald_plan_create_box(box, int(n), float(tol), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        p = ewald_params()
        _check(_lib.ewald_plan_query(self._h, ctypes.byref(p)))
        self.params = p
        self.n = int(n)
        self.L = float(L) if cube else tuple(float(v) for v in box)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ewald_plan_destroy(h)
            self._h = None

    def _stream(self):
        return ctypes.c_void_p(self._torch.cuda.current_stream(self.device).cuda_stream)

    def eval(self, x, rho, phi=None, force=None, energy=True):
        """phi (n,), F (n,3), E for device tensors x (n,3) and rho (n,) (float64, contiguous)."""
        torch = self._torch
        x = x.to(device=self.device, dtype=torch.float64).contiguous()
        rho = rho.to(device=self.device, dtype=torch.float64).contiguous()
        if x.shape != (self.n, 3) or rho.shape != (self.n,):
            raise ValueError("x must be (n,3) and rho (n,) with n = %d" % self.n)
        if phi is None:
            phi = torch.empty(self.n, dtype=torch.float64, device=self.device)
        if force is None:
            force = torch.empty(self.n, 3, dtype=torch.float64, device=self.device)
        e = ctypes.c_double(0.0)
        _check(_lib.ewald_eval(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                               ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                               ctypes.byref(e) if energy else None, self._stream()))
        return phi, force, (e.value if energy else None)

    def eval_host(self, x, rho, phi=None, force=None):
        """Same evaluation from host (NumPy) buffers; copies run inside the library call.  phi (n,) and
        force (n,3) may be caller-owned float64 arrays (page-locked ones make the copies back faster)."""
        x = _f64(x, (self.n, 3))
        rho = _f64(rho, (self.n,))
        phi = _out(phi, (self.n,))
        F = _out(force, (self.n, 3))
        e = ctypes.c_double(0.0)
        _check(_lib.ewald_eval_host(self._h, _ptr(x), _ptr(rho), _ptr(phi), _ptr(F), ctypes.byref(e),
                                    self._stream()))
        return phi, F, e.value

    def check(self):
        _check(_lib.ewald_check(self._h, self._stream()))

    STAGES = ("sort", "spread", "halo", "fft_fwd", "scale", "fft_inv", "interp", "short", "energy")

    def profile(self, enable=True, serial=False):
        """Per-stage CUDA events on (serial: with the real-space sum and Alg. 2 serialised) or off."""
        _check(_lib.ewald_profile(self._h, (2 if serial else 1) if enable else 0))

    def profile_read(self):
        """Summed milliseconds per stage over the evaluations recorded since profile(True)."""
        ms = np.zeros(len(self.STAGES))
        cnt = ctypes.c_int(0)
        _check(_lib.ewald_profile_read(self._h, _ptr(ms), ctypes.byref(cnt)))
        return dict(zip(self.STAGES, ms.tolist())), cnt.value

    def debug_grid(self, which):
        out = np.empty(tuple(self.params.grid))
        _check(_lib.ewald_debug_grid(self._h, int(which), _ptr(out)))
        return out


class _EwaldEnergy:
    """torch.autograd.Function: E(x, rho) with dE/dx = -F and dE/drho = phi (exact for the discrete operator)."""

    @staticmethod
    def build():
        import torch

        class EwaldEnergy(torch.autograd.Function):
            @staticmethod
            def forward(ctx, x, rho, plan):
                phi, F, E = plan.eval(x.detach(), rho.detach())
                ctx.save_for_backward(phi, F)
                return torch.tensor(E, dtype=torch.float64, device=x.device)

            @staticmethod
            def backward(ctx, gE):
                phi, F = ctx.saved_tensors
                return -gE * F, gE * phi, None

        return EwaldEnergy


def energy(x, rho, plan):
    """Differentiable Ewald energy (PyTorch autograd)."""
    global _ENERGY_FN
    try:
        fn = _ENERGY_FN
    except NameError:
        fn = _ENERGY_FN = _EwaldEnergy.build()
    return fn.apply(x, rho, plan)


class BatchPlan:
    """Independent systems evaluated by one call (C ABI: ewald_plan_batch_create / ewald_eval_batch).

    ``Ls`` and ``ns`` give each system's box edge and particle count; all share ``tol`` and the
    ewald_opts keywords.  ``eval`` takes the systems' rows concatenated in order.
    """

    def __init__(self, Ls, ns, tol, precision="fp64", **opts):
        import torch  # device memory and streams only
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("PSWF Ewald plans need a CUDA device (no CPU fallback)")
        torch.cuda.init()
        self.device = torch.device("cuda", torch.cuda.current_device())
        Ls = np.ascontiguousarray(Ls, dtype=np.float64)
        ns = np.ascontiguousarray(ns, dtype=np.int64)
        if Ls.shape != ns.shape or Ls.ndim != 1:
            raise ValueError("Ls and ns must be 1-D arrays of equal length")
        self.nsys = len(ns)
        self.offsets = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        o = make_opts(precision=precision, **opts)
        h = ctypes.c_void_p()
        _check(_lib.ewald_plan_batch_create(self.nsys, Ls.ctypes.data_as(ctypes.c_void_p),
                                            ns.ctypes.data_as(ctypes.c_void_p), float(tol), ctypes.byref(o),
                                            ctypes.byref(h)))
        self._h = h
        p = ewald_params()
        _check(_lib.ewald_plan_query(self._h, ctypes.byref(p)))
        self.params0 = p

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ewald_plan_destroy(h)
            self._h = None

    def eval(self, x, rho, phi=None, force=None):
        """phi (N,), F (N,3) device tensors and per-system energies (NumPy) for the concatenated rows."""
        torch = self._torch
        N = int(self.offsets[-1])
        x = x.to(device=self.device, dtype=torch.float64).contiguous()
        rho = rho.to(device=self.device, dtype=torch.float64).contiguous()
        if x.shape != (N, 3) or rho.shape != (N,):
            raise ValueError("x must be (N,3) and rho (N,) with N = %d" % N)
        if phi is None:
            phi = torch.empty(N, dtype=torch.float64, device=self.device)
        if force is None:
            force = torch.empty(N, 3, dtype=torch.float64, device=self.device)
        E = np.empty(self.nsys)
        stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        _check(_lib.ewald_eval_batch(self._h, self.offsets.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                     ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                                     E.ctypes.data_as(ctypes.c_void_p), stream))
        return phi, force, E
