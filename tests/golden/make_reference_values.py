"""Writes the stored oracle values of the two large workloads (run on a CPU; calls only oracle/ and workloads).

    python tests/golden/make_reference_values.py [uniform1e5|uniform1e7|all]

* ``uniform1e5_seed0.txt``: n = 100,000 uniform neutral charges (workloads.uniform_neutral, seed 0, L = 1):
  phi and F at 256 targets (indices linspace(0, n-1, 256)) from the converged PSWF Ewald sum of the
  oracle (exact.pswf_exact: c_s = 34, r_c = L/2, k-sphere |k| <= 14), and the total energy E.  E needs
  phi at every particle; that run uses the oracle's split at r_c = L/4 (k-sphere |k| <= 28), whose
  real-space part touches ~15x fewer pairs; split independence makes the two agree to ~1e-13, which
  the script checks on the 256 targets.
* ``uniform1e7_seed0.txt``: n = 10,000,000 (same generator and seed): phi and F at 64 targets
  (linspace(0, n-1, 64)); no energy (the real-space part over all targets is out of reach on a CPU).

Format: comment lines start with '#'; 'E <value>' holds the energy; every other line is
'<index> <phi> <Fx> <Fy> <Fz>' with 17 significant digits.
"""
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402
from workloads import uniform_neutral  # noqa: E402

CASES = {"uniform1e5": (100_000, 256, True), "uniform1e7": (10_000_000, 64, False)}


def _chunk(args):
    n, targets, rc_frac = args
    x, rho, L = uniform_neutral(n, seed=0)
    phi, _, _, F = exact.pswf_exact(x, rho, L, targets=targets, rc_frac=rc_frac)
    return phi, F


def write(name, procs):
    n, ntg, with_energy = CASES[name]
    t0 = time.time()
    tg = np.linspace(0, n - 1, ntg).astype(np.int64)
    phi, F = _chunk((n, tg, 0.5))
    E = None
    if with_energy:
        # phi at every particle, in chunks over worker processes (each recomputes the structure factor)
        x, rho, L = uniform_neutral(n, seed=0)
        parts = np.array_split(np.arange(n), max(procs * 4, 1))
        with ProcessPoolExecutor(procs) as ex:
            phis = list(ex.map(_chunk, [(n, p, 0.25) for p in parts]))
        phi_all = np.concatenate([p for p, _ in phis])
        E = 0.5 * float(np.dot(rho, phi_all))
        assert np.max(np.abs(phi_all[tg] - phi)) <= 1e-11 * np.max(np.abs(phi))
    path = os.path.join(HERE, name + "_seed0.txt")
    with open(path, "w") as fh:
        fh.write("# oracle values (exact.pswf_exact: converged PSWF Ewald sum, c_s = 34, r_c = L/2)\n")
        fh.write("# workload: workloads.uniform_neutral(n=%d, seed=0), L = 1; targets linspace(0, n-1, %d)\n"
                 % (n, ntg))
        fh.write("# written by tests/golden/make_reference_values.py %s (%.0f s)\n" % (name, time.time() - t0))
        if E is not None:
            fh.write("E %.17e\n" % E)
        for i, p, f in zip(tg, phi, F):
            fh.write("%d %.17e %.17e %.17e %.17e\n" % (i, p, f[0], f[1], f[2]))
    return path


def read(name):
    """(targets, phi, F, E or None) of a stored file."""
    E, rows = None, []
    with open(os.path.join(HERE, name + "_seed0.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            if f[0] == "E":
                E = float(f[1])
            else:
                rows.append([float(v) for v in f])
    a = np.array(rows)
    return a[:, 0].astype(np.int64), a[:, 1], a[:, 2:5], E


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    procs = int(os.environ.get("PROCS", os.cpu_count() or 1))
    for nm in (CASES if which == "all" else [which]):
        print(write(nm, procs), flush=True)
