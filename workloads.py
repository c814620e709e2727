"""Seeded synthetic particle systems (inputs only; no Ewald arithmetic here).

Shared by the tests, the oracle runs and ``bench.py``.  This module imports neither
the CUDA library's package nor ``oracle``, so generating inputs never loads the
library.  Every generator uses
NumPy's PCG64 with an explicit seed and returns ``(x, rho, L)`` with ``x`` an
(n, 3) float64 array in [0, L)^3 and ``rho`` a float64 array summing to zero
(to rounding).  The shapes follow the paper's experiments (Sec. 7.1: uniform
points, charges shifted to neutrality) and the MD-like systems the library
targets.
"""
import numpy as np


def _neutralise(rho):
    rho = np.asarray(rho, dtype=np.float64)
    return rho - rho.mean()


def uniform_alternating(n=1000, L=1.0, seed=0):
    """n uniform points, rho_j = +1, -1, +1, ... (n even gives exact neutrality)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.random((n, 3)) * L
    rho = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    if n % 2:
        rho = _neutralise(rho)
    return x, rho, float(L)


def uniform_neutral_box(n, box=(1.0, 1.0, 2.0), seed=0):
    """n uniform points in the cuboid prod_d [0, box_d); rho ~ U[-1, 1] minus its mean."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.random((n, 3)) * np.asarray(box, dtype=np.float64)
    return x, _neutralise(rng.uniform(-1.0, 1.0, n)), tuple(float(b) for b in box)


def uniform_neutral(n=100_000, L=1.0, seed=0, dist="uniform"):
    """n uniform points; rho ~ U[-1, 1] (or N(0,1)) minus its mean."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.random((n, 3)) * L
    if dist == "uniform":
        rho = rng.uniform(-1.0, 1.0, n)
    else:
        rho = rng.standard_normal(n)
    return x, _neutralise(rho), float(L)


def nacl_lattice(cells=4, L=1.0):
    """Rock salt: cells^3 conventional cubic cells of edge a = L/cells, 8 ions each.

    Na+ on the fcc sites (0,0,0) + face centres, Cl- displaced by (a/2, 0, 0).
    All coordinates are exact multiples of a/2.  Nearest-neighbour distance a/2.
    """
    a = L / cells
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    pts, q = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                o = np.array([i, j, k], dtype=np.float64)
                for f in fcc:
                    pts.append((o + f) * a)
                    q.append(1.0)
                    pts.append((o + f + np.array([0.5, 0.0, 0.0])) * a)
                    q.append(-1.0)
    x = np.mod(np.array(pts), L)
    return x, np.array(q), float(L)


def water_box(n_mol=33_000, density=33.4, seed=0, min_dist=0.12):
    """Rigid 3-site water-like molecules in a cubic box (nm units, charges in e).

    O at -0.8476, two H at +0.4238, O-H 0.1 nm, HOH 109.47 deg; O sites drawn
    without replacement from a cubic lattice with jitter, orientations uniform.
    Orientations of molecules with an intermolecular site pair closer than
    ``min_dist`` are redrawn (periodic k-d tree query) until none is left.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    L = (n_mol / density) ** (1.0 / 3.0)
    side = int(np.ceil(n_mol ** (1.0 / 3.0)))
    spacing = L / side
    sites = rng.choice(side ** 3, size=n_mol, replace=False)
    ijk = np.stack(np.unravel_index(sites, (side,) * 3), axis=1).astype(np.float64)
    O = (ijk + 0.5) * spacing + rng.uniform(-0.03, 0.03, (n_mol, 3))
    th = np.deg2rad(109.47) / 2.0
    body = np.array([[0.0, 0.0, 0.0],
                     [0.1 * np.sin(th), 0.0, 0.1 * np.cos(th)],
                     [-0.1 * np.sin(th), 0.0, 0.1 * np.cos(th)]])

    def rand_rot(k):
        qv = rng.standard_normal((k, 4))
        qv /= np.linalg.norm(qv, axis=1, keepdims=True)
        w, xq, yq, zq = qv.T
        return np.stack([
            np.stack([1 - 2 * (yq * yq + zq * zq), 2 * (xq * yq - zq * w), 2 * (xq * zq + yq * w)], -1),
            np.stack([2 * (xq * yq + zq * w), 1 - 2 * (xq * xq + zq * zq), 2 * (yq * zq - xq * w)], -1),
            np.stack([2 * (xq * zq - yq * w), 2 * (yq * zq + xq * w), 1 - 2 * (xq * xq + yq * yq)], -1),
        ], 1)

    from scipy.spatial import cKDTree

    Rm = rand_rot(n_mol)
    pos = O[:, None, :] + np.einsum('mij,sj->msi', Rm, body)
    # redraw the orientations of molecules with an intermolecular site pair closer than min_dist
    for _ in range(200):
        flat = np.mod(pos.reshape(-1, 3), L)
        pairs = cKDTree(flat, boxsize=L).query_pairs(min_dist, output_type='ndarray')
        mol = np.arange(3 * n_mol) // 3
        if len(pairs):
            pairs = pairs[mol[pairs[:, 0]] != mol[pairs[:, 1]]]
        if len(pairs) == 0:
            break
        idx = np.unique(mol[pairs.ravel()])
        Rm[idx] = rand_rot(len(idx))
        pos[idx] = O[idx, None, :] + np.einsum('mij,sj->msi', Rm[idx], body)
    x = np.mod(pos.reshape(-1, 3), L)
    q = np.tile(np.array([-0.8476, 0.4238, 0.4238]), n_mol)
    return x, q, float(L)


def batched_systems(nsys=256, seed=0, density=100.0, nmin=500, nmax=20_000):
    """Independent neutral uniform systems, n log-uniform in [nmin, nmax], L = (n/density)^(1/3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax), nsys))).astype(np.int64)
    out = []
    for i, n in enumerate(ns):
        L = (n / density) ** (1.0 / 3.0)
        x, rho, _ = uniform_neutral(int(n), L=L, seed=seed * 100_003 + i + 1)
        out.append((x, rho, float(L)))
    return out
