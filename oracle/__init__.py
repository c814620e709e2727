"""Plain FP64 CPU oracle for PSWF fast Ewald summation (test infrastructure only).

This package is NOT part of the product path.  Only the test suite, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library under ``paper_2602_16591_gb300``.

Modules
-------
pswf      first prolate spheroidal wave function psi_0^c: dense symmetric
          eigensolver on the Legendre-basis matrix of the ODE (Sec. 2.4, App. B).
split     PSWF mollifier, split function Phi, residual R, mollifier transform
          (Sec. 4.1-4.2, Table 1) and the classical Gaussian split (Example 1).
exact     the converged Ewald sum (Sec. 3.1, Alg. 1 with converged k-range plus
          the real-space sum and self term), brute-force lattice sums.
alg2      Alg. 2 (fast Fourier-space sum) restated step by step with exact psi.
params    Alg. 3 parameter selection (Sec. 6) as printed, with the readings it needs
          (relative tolerance, Lambert-W branches, instantiation after rounding).

Parity status: every public function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (identities, library special cases, the NaCl Madelung
constant, brute-force lattice sums, split independence, the paper's Table 3).
The closed-form error models of Sec. 5 are approximations by nature; the tests
compare them with measured errors only within the factor the paper reports.

Nothing here imports the CUDA library's package.  Callers take their seeded inputs
from the top-level ``workloads`` module, which holds no arithmetic of the method and
does not load the library either.
"""
