"""Time-slice contractions of the stochastic estimator (oracle; test
infrastructure only).

Sec. 5, Eq. C_stoch2: for one noise source eta with support on time slice
y0, the estimator of the isovector vector correlator between levels i, j is

    G_ij^n(x0, y0) = -(1 / (3 L^3)) sum_{k=1}^{3} sum_{x: time slice x0}
                     < (S_j gamma5 gamma_k^dag eta)(x), gamma5 gamma_k (S_i eta)(x) >

(lattice units a = 1; <u, v> = sum over spin and colour of conj(u) v).  The
inputs here are the solved fields: a_k = S_j gamma5 gamma_k^dag eta for
k = 1, 2, 3 and b = S_i eta.  ``slice_correlator`` evaluates the sum above
for every x0 directly from that definition.

Eq. tmr defines the correlator itself through the full propagator,

    C(x0, y0) = -(1 / (3 L^3)) sum_k sum_{x in x0, y in y0} tr{S(x, y) gamma_k S(y, x) gamma_k},

which ``correlator_from_propagator`` evaluates from a dense S.  Summing the
estimator over the 12 spin-colour point sources at every y of slice y0
reproduces C exactly (gamma5-hermiticity S(y, x) = gamma5 S(x, y)^dag
gamma5); the pin in tests/test_oracle_contract.py checks that identity.

Eq. timetrans: the translation average G(t) = (1 / L0) sum_{y0} C(t + y0, y0)
(``translation_average``), with x0 taken modulo L0.

Sec. "Exact estimator on the coarsest grid" (Eq. G_LL:exact): on a coarse
level small enough to invert densely, the level's contribution to G(t) is

    G(t) = -(1 / (3 L0 L^3)) sum_k sum_{y0} tr{ Gam_k(y0 + t) Q_c^-1 Gam_k(y0) Q_c^-1 }

with Q_c = g5hat D_c the Hermitian coarse operator and the coarse matrices
Gam_k(x0) = calR gamma5 gamma_k P_{x0} calT (P_{x0} keeps fine time slice
x0), the open-index analogue of Eq. coarse:gamma.  On level 1 they are
block-diagonal over coarse sites: Gam_k(x0)[y] = sum_{x in B_y, time x0}
phi_i(x)^dag gamma5 gamma_k phi_j(x); an inner-level transfer keeps them
block-diagonal, Gam(x0)[y] on level l + 1 = (V_{l+1} / V_l) sum_{z in B_y}
Gam(x0)[z] on level l.  ``exact_coarse_correlator`` evaluates the trace
formula from the dense inverse; the pin in tests/test_oracle_exact.py
compares it with C_11 of Eq. lma:ee summed from the dense coarse-level
propagator calT D_c^-1 calR (App. chirality) on the fine lattice.
"""
from __future__ import annotations

import numpy as np

from . import dirac as _d


def gamma5_gamma(k: int) -> np.ndarray:
    """gamma5 gamma_k (k = 1, 2, 3), a 4x4 spin matrix."""
    return _d.gamma5() @ _d.gammas()[k]


def spin_apply(M: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(M psi)(x) for a 4x4 spin matrix M and a field (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", M, psi)


def slice_correlator(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """-(1 / (3 L^3)) sum_k sum_{x in x0} <a_k(x), gamma5 gamma_k b(x)> for
    every time slice x0.  a: (3, L0, L1, L2, L3, 4, 3), b: (L0, L1, L2, L3,
    4, 3).  Returns complex (L0,)."""
    L0 = b.shape[0]
    L3vol = b.shape[1] * b.shape[2] * b.shape[3]
    out = np.zeros(L0, dtype=np.complex128)
    for k in range(1, 4):
        gb = spin_apply(gamma5_gamma(k), b)
        for x0 in range(L0):
            out[x0] += np.vdot(a[k - 1][x0].reshape(-1), gb[x0].reshape(-1))
    return -out / (3.0 * L3vol)


def correlator_from_propagator(S: np.ndarray, L, y0: int) -> np.ndarray:
    """C(x0, y0) of Eq. tmr for every x0 from the dense propagator S
    (V*12 x V*12, site-major then spin then colour)."""
    L = tuple(int(v) for v in L)
    V = int(np.prod(L))
    L3vol = V // L[0]
    g = _d.gammas()
    Sb = S.reshape(V, 4, 3, V, 4, 3)
    out = np.zeros(L[0], dtype=np.complex128)
    ys = [y0 * L3vol + s for s in range(L3vol)]
    for x0 in range(L[0]):
        for xs in range(L3vol):
            x = x0 * L3vol + xs
            for y in ys:
                Sxy = Sb[x, :, :, y, :, :].reshape(12, 12)  # (s c) x (t d)
                Syx = Sb[y, :, :, x, :, :].reshape(12, 12)
                for k in range(1, 4):
                    G = np.kron(g[k], np.eye(3))
                    out[x0] += np.trace(Sxy @ G @ Syx @ G)
    return -out / (3.0 * L3vol)


def translation_average(C: np.ndarray) -> np.ndarray:
    """G(t) = (1 / L0) sum_{y0} C[(t + y0) mod L0, y0] for C of shape (L0, L0)
    indexed [x0, y0]."""
    L0 = C.shape[0]
    return np.array([sum(C[(t + y0) % L0, y0] for y0 in range(L0)) / L0 for t in range(L0)])


def coarse_gamma5_gamma(phi: np.ndarray, L, b, k: int) -> np.ndarray:
    """Gam_k(x0) on level 1 for every fine time slice x0: array (L0, V1, n, n),
    block y of slice x0 = sum over the sites x of B_y on slice x0 of
    phi_i(x)^dag gamma5 gamma_k phi_j(x) (zero when B_y misses x0); phi as in
    ``multigrid.build_basis``."""
    from . import lattice as _lat
    L = tuple(int(v) for v in L)
    V1, _, nv = phi.shape[:3]
    n = 2 * nv
    sites = _lat.block_sites(L, b)  # (V1, nB)
    x0_of = _lat.coords(L)[:, 0]
    G5k = gamma5_gamma(k)
    out = np.zeros((L[0], V1, n, n), dtype=np.complex128)
    ph = phi.reshape(V1, n, phi.shape[3], 4, 3)  # (y, i, site-in-block, spin, colour)
    for y in range(V1):
        gphi = np.einsum("st,jktc->jksc", G5k, ph[y])
        for kk, site in enumerate(sites[y]):
            x0 = x0_of[site]
            out[x0, y] += np.einsum("isc,jsc->ij", np.conj(ph[y][:, kk]), gphi[:, kk])
    return out


def coarse_gamma_next(Gam: np.ndarray, Lb, b) -> np.ndarray:
    """Gam(x0) on the next level: (V_{l+1} / V_l) times the sum of the blocks
    of the level-l sites of each next-level block."""
    from . import lattice as _lat
    Lb2 = _lat.block_grid(Lb, b)
    V1, V2 = _lat.volume(Lb), _lat.volume(Lb2)
    blk = _lat.block_of_site(Lb, b)
    out = np.zeros((Gam.shape[0], V2) + Gam.shape[2:], dtype=np.complex128)
    for z in range(V1):
        out[:, blk[z]] += Gam[:, z]
    return out * (V2 / V1)


def exact_coarse_correlator(Dhat: np.ndarray, Lb, Gams, L) -> tuple:
    """(C, G): C[x0, y0] = -(1 / (3 L^3)) sum_k tr{Gam_k(y0) Q^-1 Gam_k(x0) Q^-1}
    and its translation average G(t) (Eq. G_LL:exact), Q = g5hat D_c dense,
    Gams[k-1] = Gam_k as from ``coarse_gamma5_gamma`` / ``coarse_gamma_next``."""
    from . import multigrid as _mg
    L = tuple(int(v) for v in L)
    n = Dhat.shape[2]
    V1 = Dhat.shape[1]
    g5 = np.tile(_mg.coarse_gamma5(n // 2), V1)
    Qi = np.linalg.inv(g5[:, None] * _mg.dense_coarse(Dhat, Lb))
    L0 = L[0]
    C = np.zeros((L0, L0), dtype=np.complex128)
    for Gam in Gams:
        dense = [np.zeros((V1 * n, V1 * n), dtype=np.complex128) for _ in range(L0)]
        for t in range(L0):
            for y in range(V1):
                dense[t][y * n:(y + 1) * n, y * n:(y + 1) * n] = Gam[t, y]
        for x0 in range(L0):
            for y0 in range(L0):
                C[x0, y0] += np.trace(dense[y0] @ Qi @ dense[x0] @ Qi)
    C *= -1.0 / (3.0 * (int(np.prod(L)) // L0))
    return C, translation_average(C)
