"""Pins of the oracle's converged Ewald sum (Sec. 3.1) against facts independent of the split."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import exact
from workloads import nacl_lattice, uniform_neutral


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def small_system():
    x, rho, L = uniform_neutral(40, L=1.0, seed=3, dist="normal")
    return x, rho, L


def test_split_independence(small_system):
    """The total does not depend on the split: two PSWF cutoffs and the Gaussian split agree."""
    x, rho, L = small_system
    a = exact.pswf_exact(x, rho, L, cs=34.0, rc_frac=0.5)
    b = exact.pswf_exact(x, rho, L, cs=34.0, rc_frac=0.3)
    g = exact.gaussian_exact(x, rho, L, xi=6.0)
    for o in (b, g):
        assert _rel(o[0], a[0]) <= 1e-13
        assert _rel(o[3], a[3]) <= 1e-12
        assert abs(o[2] - a[2]) <= 1e-12 * abs(a[2])


def test_split_independence_detects_wrong_self_term(small_system):
    """A plausible mistake (self term with lambda_0 dropped) is caught by the same comparison."""
    x, rho, L = small_system
    from oracle.split import PSWFSplit
    sp = PSWFSplit(34.0, 0.5)
    phi, _, _, _ = exact.pswf_exact(x, rho, L)
    bad = phi + sp.self_coeff() * rho - 2.0 / 0.5 * rho
    g = exact.gaussian_exact(x, rho, L)
    assert _rel(bad, g[0]) > 1e-3


def test_nacl_madelung():
    M = float(read_golden("nacl_madelung.txt")[0][1])
    x, q, L = nacl_lattice(cells=4, L=1.0)
    phi, grad, E, F = exact.pswf_exact(x, q, L)
    d = L / 8.0
    assert np.allclose(phi, -q * M / d, rtol=1e-12, atol=0)
    assert abs(E - (-len(q) * M / (2 * d))) <= 1e-11 * abs(E)
    assert np.max(np.abs(F)) <= 1e-11 * M / d ** 2


def test_stored_values_are_the_oracles():
    """The stored oracle values of the 1e5 bench workload (tests/golden/uniform1e5_seed0.txt, written by
    tests/golden/make_reference_values.py) are reproduced by the oracle as it stands at three of their
    targets: the GPU parity tests that read them compare against the present oracle, not a stale copy."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_reference_values as stored
    tg, phi, F, _ = stored.read("uniform1e5")
    sel = np.array([0, 131, len(tg) - 1])
    x, rho, L = uniform_neutral(100_000, seed=0)
    p, _, _, f = exact.pswf_exact(x, rho, L, targets=tg[sel])
    assert np.max(np.abs(p - phi[sel])) <= 1e-12 * np.max(np.abs(phi))
    assert np.max(np.abs(f - F[sel])) <= 1e-12 * np.max(np.abs(F))


def test_madelung_value_by_benson_series():
    """The stored rock-salt constant against an independent route: Benson's series
    M = 12 pi sum_{m, n odd > 0} sech^2((pi/2) sqrt(m^2 + n^2)), which converges like exp(-pi m) and
    involves no Ewald split, so the NaCl pin above rests on more than a remembered number."""
    M = float(read_golden("nacl_madelung.txt")[0][1])
    odd = np.arange(1, 41, 2, dtype=np.float64)
    mm, nn = np.meshgrid(odd, odd)
    benson = 12 * np.pi * np.sum(1.0 / np.cosh(0.5 * np.pi * np.sqrt(mm * mm + nn * nn)) ** 2)
    assert abs(benson - M) <= 1e-12


def _extrapolate(vals, Ns, powers=(2, 3, 4)):
    """Least-squares fit v(N) = v_inf + sum_p a_p N^-p over the shell sums; returns v_inf."""
    A = np.array([[1.0] + [float(N) ** -p for p in powers] for N in Ns])
    V = np.array([np.ravel(v) for v in vals])
    return np.linalg.lstsq(A, V, rcond=None)[0][0].reshape(np.shape(vals[0]))


@pytest.mark.parametrize("seed", [1, 2])
def test_bruteforce_lattice_sum(seed):
    """Dipole-free neutral cells: the cubic-shell replica sum of 1/r converges to the
    Ewald potential minus the constant (2 pi/(3V)) sum_j rho_j |x_j - c|^2 (a derivation
    of this library; no gradient), so phi and forces are pinned together."""
    rng = np.random.default_rng(seed)
    c = np.full(3, 0.5)
    a = rng.uniform(-0.3, 0.3, (2, 3))
    x = np.array([c + a[0], c - a[0], c + a[1], c - a[1]])
    rho = np.array([1.0, 1.0, -1.0, -1.0])
    ref = exact.pswf_exact(x, rho, 1.0)
    Ns = (8, 12, 16, 24, 32)
    sums = [exact.lattice_shell_sum(x, rho, 1.0, N) for N in Ns]
    const = 2 * np.pi / 3.0 * np.sum(rho * np.sum((x - c) ** 2, axis=1))
    phi = _extrapolate([s[0] for s in sums], Ns) + const
    grad = _extrapolate([s[1] for s in sums], Ns)
    assert np.max(np.abs(phi - ref[0])) <= 1e-7 * np.max(np.abs(ref[0]))
    assert np.max(np.abs(grad - ref[1])) <= 1e-7 * np.max(np.abs(ref[1]))


@pytest.mark.parametrize("seed", [1, 2])
def test_bruteforce_lattice_sum_with_dipole(seed):
    """General neutral cells (dipole D = sum_j rho_j x_j != 0): the cubic-shell replica sum is the
    sum of a macroscopic cube in vacuum, whose depolarisation factor is 1/3 by symmetry, so it exceeds
    the Ewald (conducting-boundary) potential by the surface term (4 pi/(3V)) D . x_i and the
    second-moment constant -(2 pi/(3V)) sum_j rho_j |x_j|^2 (the two together do not depend on the
    origin), the field by (4 pi/(3V)) D, and the energy by (2 pi/(3V)) |D|^2 (a derivation of this
    library, checked here; dropping the surface term, flipping its sign or halving it misses by 5-90%)."""
    rng = np.random.default_rng(seed)
    x = rng.random((5, 3))
    rho = rng.uniform(-1.0, 1.0, 5)
    rho -= rho.mean()
    D = rho @ x
    V = 1.0
    ref = exact.pswf_exact(x, rho, 1.0)
    Ns = (8, 12, 16, 24, 32)
    sums = [exact.lattice_shell_sum(x, rho, 1.0, N) for N in Ns]
    phi_shell = _extrapolate([s[0] for s in sums], Ns)
    grad_shell = _extrapolate([s[1] for s in sums], Ns)
    phi = phi_shell - 4 * np.pi / (3 * V) * (x @ D) + 2 * np.pi / (3 * V) * np.sum(rho * np.sum(x * x, axis=1))
    grad = grad_shell - 4 * np.pi / (3 * V) * D
    assert np.linalg.norm(D) > 0.1
    assert np.max(np.abs(phi - ref[0])) <= 1e-7 * np.max(np.abs(ref[0]))
    assert np.max(np.abs(grad - ref[1])) <= 1e-7 * np.max(np.abs(ref[1]))
    E_shell = 0.5 * float(rho @ phi_shell)
    assert abs(E_shell - (ref[2] + 2 * np.pi / (3 * V) * float(D @ D))) <= 1e-7 * abs(ref[2])


def test_bruteforce_catches_a_flipped_structure_factor_phase(monkeypatch):
    """A planted mistake in the k-space sum: rho-hat with the sign of its phase flipped (its conjugate).
    The centrosymmetric NaCl lattice has a real structure factor and does not notice it; the brute-force
    lattice sum, which shares no code with the k-space sum, does (so does split independence, whose two
    splits weight the wrong modes differently)."""
    rng = np.random.default_rng(1)
    x = rng.random((5, 3))
    rho = rng.uniform(-1.0, 1.0, 5)
    rho -= rho.mean()
    D = rho @ x
    Ns = (8, 12, 16, 24, 32)
    sums = [exact.lattice_shell_sum(x, rho, 1.0, N) for N in Ns]
    phi_bf = _extrapolate([s[0] for s in sums], Ns) - 4 * np.pi / 3 * (x @ D) \
        + 2 * np.pi / 3 * np.sum(rho * np.sum(x * x, axis=1))
    good = exact.pswf_exact(x, rho, 1.0)[0]
    orig = exact.structure_factor
    monkeypatch.setattr(exact, "structure_factor", lambda *a, **k: np.conj(orig(*a, **k)))
    bad = exact.pswf_exact(x, rho, 1.0)[0]
    scale = np.max(np.abs(phi_bf))
    assert np.max(np.abs(good - phi_bf)) <= 1e-7 * scale
    assert np.max(np.abs(bad - phi_bf)) > 1e-3 * scale


def test_translation_invariance(small_system):
    x, rho, L = small_system
    a = exact.pswf_exact(x, rho, L)
    b = exact.pswf_exact(np.mod(x + np.array([0.31, -0.72, 0.45]), L), rho, L)
    assert _rel(b[0], a[0]) <= 1e-13 and _rel(b[3], a[3]) <= 1e-12


def test_scaling_law(small_system):
    """eq. phinondim: phi(s x; s L) = phi(x; L)/s, forces scale as 1/s^2."""
    x, rho, L = small_system
    s = 3.7
    a = exact.pswf_exact(x, rho, L)
    b = exact.pswf_exact(s * x, rho, s * L)
    assert _rel(b[0], a[0] / s) <= 1e-13
    assert _rel(b[3], a[3] / s ** 2) <= 1e-12


def test_forces_sum_to_zero(small_system):
    x, rho, L = small_system
    _, _, _, F = exact.pswf_exact(x, rho, L)
    assert np.max(np.abs(F.sum(axis=0))) <= 1e-12 * np.max(np.abs(F)) * len(rho)


def test_rms_potential_matches_kappa():
    """RMS(phi) ~ sqrt(kappa) ||rho|| / L for uniform neutral charges (the relative-tol reading)."""
    from oracle.params import KAPPA
    r = []
    for seed in range(3):
        x, rho, L = uniform_neutral(600, seed=seed)
        phi = exact.pswf_exact(x, rho, L)[0]
        r.append(np.sqrt(np.mean(phi ** 2)) / np.linalg.norm(rho))
    assert abs(np.mean(r) / np.sqrt(KAPPA) - 1.0) < 0.15


# ------------------------------------------------------------------ cuboid boxes (Remark, Sec. 6.1) --
def _neutral(n, seed, Lv):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 3)) * np.asarray(Lv)
    q = rng.uniform(-1, 1, n)
    return x, q - q.mean()


@pytest.mark.parametrize("reps", [(1, 1, 2), (3, 1, 1)])
def test_cuboid_supercell_reproduces_cube(reps):
    """A cubic system replicated into a cuboid supercell has the same periodic potential: every copy
    of particle i sees phi_i of the cube (and the same force); the energy scales with the copies."""
    x, q = _neutral(30, 4, (1.0, 1.0, 1.0))
    phi, grad, E, F = exact.pswf_exact(x, q, 1.0)
    shifts = np.array([(a, b, c) for a in range(reps[0]) for b in range(reps[1]) for c in range(reps[2])], float)
    xs = np.concatenate([x + s for s in shifts])
    qs = np.tile(q, len(shifts))
    phis, grads, Es, Fs = exact.pswf_exact(xs, qs, np.array(reps, float))
    n = len(q)
    for c in range(len(shifts)):
        assert np.max(np.abs(phis[c * n:(c + 1) * n] - phi)) <= 1e-11 * np.max(np.abs(phi))
        assert np.max(np.abs(Fs[c * n:(c + 1) * n] - F)) <= 1e-10 * np.max(np.abs(F))
    assert abs(Es - len(shifts) * E) <= 1e-11 * abs(len(shifts) * E)


def test_cuboid_split_independence():
    """Two PSWF cutoffs and the Gaussian split give the same Ewald sum in a cuboid (1, 1.3, 0.8)."""
    Lv = (1.0, 1.3, 0.8)
    x, q = _neutral(40, 5, Lv)
    a = exact.pswf_exact(x, q, Lv, rc_frac=0.5)
    b = exact.pswf_exact(x, q, Lv, rc_frac=0.35)
    c = exact.gaussian_exact(x, q, Lv)
    for r in (b, c):
        assert np.max(np.abs(r[0] - a[0])) <= 1e-12 * np.max(np.abs(a[0]))
        assert np.max(np.abs(r[3] - a[3])) <= 1e-11 * np.max(np.abs(a[3]))
        assert abs(r[2] - a[2]) <= 1e-12 * abs(a[2])


def test_cuboid_translation_invariance_and_wrap():
    Lv = np.array([0.9, 1.2, 1.5])
    x, q = _neutral(25, 6, Lv)
    a = exact.pswf_exact(x, q, Lv)
    b = exact.pswf_exact(x + np.array([0.31, -2.7, 4.1]), q, Lv)
    assert np.max(np.abs(b[0] - a[0])) <= 1e-12 * np.max(np.abs(a[0]))
    assert np.max(np.abs(np.sum(a[3], axis=0))) <= 1e-11 * np.max(np.abs(a[3]))
