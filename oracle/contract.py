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
