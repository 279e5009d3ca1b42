"""Plain, slow FP64 CPU oracle for the multigrid low-mode-averaging hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it; the two meet only through
the seeded input generators in ``synthetic/``.

Every function evaluates a definition of arXiv:2412.06347 (Gruber, Harris,
Krstic Marinkovic, "Multigrid low-mode averaging") directly in complex128,
without blocking, fusion or reordering beyond what the definition states:

* ``lattice``   -- the lattice, its periodic neighbours and the regular block
                   decomposition of Sec. 3 (Eqs. block_decomp, block_def,
                   block_grid).
* ``dirac``     -- gamma matrices, the clover field strength and the
                   O(a)-improved Wilson-clover operator D and Q = gamma5 D of
                   Sec. 2 (the operator whose form the paper leaves to the
                   "O(a)-improved Wilson" ensembles of Tab. ensembles).
* ``multigrid`` -- test-vector smoothing, the chirality-split block basis of
                   Eq. mg_basis with Gram-Schmidt, the restrictor R0 (Eq.
                   res_mg), prolongator T0 (Eq. pro_mg), and the coarse
                   operator D1 = R0 D T0 as a nine-slot stencil (Sec. 4,
                   Fig. A); the inner-level transfers R_l / T_l with
                   sqrt(V_{l+1} / V_l), the recursive D_{l+1} = R_l D_l T_l
                   and the multilevel pieces (Sec. "Multigrid
                   decompositions").
* ``solvers``   -- CG on the normal equations, dense solves, the
                   propagator pieces S1 = T Q1^-1 R gamma5 and S0 = S - S1
                   (Sec. 2, App. chirality), the FP64 residual evaluated in
                   time slabs, and the even-odd (Schur) decomposition of a
                   dense operator.
* ``contract``  -- the time-slice contraction of the stochastic estimator
                   (Sec. 5, Eq. C_stoch2), the correlator from a dense
                   propagator (Eq. tmr), the translation average (Eq.
                   timetrans), and the exact estimator on a coarse level
                   with its coarse gamma5 gamma_k matrices (Eq. G_LL:exact,
                   Eq. coarse:gamma).

Parity pins (tests/test_oracle_*.py) tie each part to facts that do not come
from this package: the free-field momentum-space spectrum, an abelian
constant-field clover, gamma5-hermiticity, gauge covariance, QR factorisation,
brute-force dense matrices, dense LU inverses, the eigenvalue alignment of
App. spectra, the Krylov-space minimiser that CG reaches, the block-LU
determinant identity, and fine-lattice definitions evaluated densely.  No
function here is "parity unpinned".
"""
from . import lattice, dirac, multigrid, solvers, contract  # noqa: F401
