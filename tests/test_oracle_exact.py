"""Pins of the oracle's exact coarsest-level estimator (Sec. "Exact estimator
on the coarsest grid", Eq. G_LL:exact; Eq. coarse:gamma) against the fine-
lattice definitions on 4^4: the coarse gamma5 gamma_k matrices equal
calR (gamma5 gamma_k P_x0) calT built from dense fine matrices, and the trace
formula on the coarse space equals C_ll of Eq. lma:ee evaluated from the dense
coarse-level propagator S_l = calT D_l^-1 calR on the fine lattice (App.
chirality: calT Q_l^-1 calR gamma5 = calT D_l^-1 calR), on every level of a
three-level chain down to the one-site grid."""
import numpy as np
import pytest

import synthetic
from oracle import contract as K
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG

L, B0, NV = (4, 4, 4, 4), (2, 2, 2, 2), 2
BLOCKS = [(2, 2, 1, 1), (1, 1, 2, 2)]
KAPPA, CSW = 0.124, 1.4


@pytest.fixture(scope="module")
def chain():
    U = synthetic.gauge_links(L, 0.3, 71)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, NV, 72), KAPPA, CSW, B0, 3)
    Lbs = [lat.block_grid(L, B0)]
    Dh = [MG.coarse_operator(U, phi, KAPPA, CSW, B0)]
    Gams = [[K.coarse_gamma5_gamma(phi, L, B0, k) for k in (1, 2, 3)]]
    Tc = [MG.dense_prolongator(phi, L, B0)]
    for b in BLOCKS:
        Dh.append(MG.coarse_operator_next(Dh[-1], Lbs[-1], b))
        Gams.append([K.coarse_gamma_next(G, Lbs[-1], b) for G in Gams[-1]])
        Tc.append(Tc[-1] @ np.kron(MG.dense_restrict_level(Lbs[-1], b), np.eye(2 * NV)).T)
        Lbs.append(lat.block_grid(Lbs[-1], b))
    M = D.dense_dirac(U, KAPPA, CSW)
    return dict(U=U, phi=phi, Lbs=Lbs, Dh=Dh, Gams=Gams, Tc=Tc, M=M)


def slice_projector(x0):
    """P_x0 on the fine space (12 V), site-major."""
    V = lat.volume(L)
    p = (lat.coords(L)[:, 0] == x0).astype(float)
    return np.diag(np.repeat(p, 12))


def test_coarse_gamma_matrices_are_galerkin(chain):
    V = lat.volume(L)
    for l in range(3):
        Tc, Lb = chain["Tc"][l], chain["Lbs"][l]
        n = 2 * NV
        for k in (1, 2, 3):
            G5k = np.kron(np.eye(V), np.kron(K.gamma5_gamma(k), np.eye(3)))
            for x0 in range(L[0]):
                ref = Tc.conj().T @ G5k @ slice_projector(x0) @ Tc
                got = np.zeros_like(ref)
                for y in range(lat.volume(Lb)):
                    got[y * n:(y + 1) * n, y * n:(y + 1) * n] = chain["Gams"][l][k - 1][x0, y]
                assert np.abs(got - ref).max() < 1e-13, (l, k, x0)


def test_exact_estimator_equals_fine_definition(chain):
    M = chain["M"]
    for l in range(3):
        Tc = chain["Tc"][l]
        S = Tc @ np.linalg.solve(Tc.conj().T @ M @ Tc, Tc.conj().T)
        C_ref = np.stack([K.correlator_from_propagator(S, L, y0) for y0 in range(L[0])], axis=1)
        C, G = K.exact_coarse_correlator(chain["Dh"][l], chain["Lbs"][l], chain["Gams"][l], L)
        assert np.abs(C - C_ref).max() < 1e-12 * np.abs(C_ref).max(), l
        assert np.abs(G - K.translation_average(C_ref)).max() < 1e-12 * np.abs(C_ref).max()
        # the correlator of a Hermitian-conjugate pair of currents is real
        assert np.abs(G.imag).max() < 1e-12 * np.abs(G.real).max()
