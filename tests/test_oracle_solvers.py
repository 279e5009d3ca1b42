"""Pins of the oracle's solvers and propagator pieces (Sec. 2, App. chirality)
against dense LU inverses."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG
from oracle import solvers as S


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


@pytest.fixture(scope="module")
def dense_setup():
    L, b, nv = (4, 2, 2, 2), (2, 2, 2, 2), 3
    kappa, csw = 0.125, 1.7
    U = synthetic.gauge_links(L, 0.3, 71)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 72), kappa, csw, b, 3)
    Dhat = MG.coarse_operator(U, phi, kappa, csw, b)
    M = D.dense_dirac(U, kappa, csw)
    T = MG.dense_prolongator(phi, L, b)
    Lb = lat.block_grid(L, b)
    return dict(L=L, b=b, nv=nv, kappa=kappa, csw=csw, U=U, phi=phi, Dhat=Dhat, M=M, T=T, Lb=Lb)


def test_cgne_matches_dense_solve(dense_setup):
    s = dense_setup
    eta = synthetic.z2_noise(s["L"], 1, 3)[0]
    x, it, res = S.solve_fine(s["U"], eta, s["kappa"], s["csw"], tol=1e-12)
    assert res <= 1e-12 and it > 0
    xd = np.linalg.solve(s["M"], eta.reshape(-1))
    assert rel(x.reshape(-1), xd) < 1e-10
    assert S.true_residual(s["U"], x, eta, s["kappa"], s["csw"]) < 1e-11


def test_coarse_cgne_matches_dense_solve(dense_setup):
    s = dense_setup
    b1 = synthetic.random_coarse(lat.volume(s["Lb"]), 2 * s["nv"], 1, 9)[0]
    X, it, res = S.solve_coarse(s["Dhat"], b1, s["Lb"], tol=1e-13)
    Xd = np.linalg.solve(MG.dense_coarse(s["Dhat"], s["Lb"]), b1.reshape(-1))
    assert rel(X.reshape(-1), Xd) < 1e-10


def test_decomposition_sums_to_dense_inverse(dense_setup):
    """S = S0 + S1 with S1 = T Q1^-1 R gamma5; Galerkin identities
    R D S0 = 0 and S0 D T = 0; App. chirality: T Q1^-1 R gamma5 = T D1^-1 R."""
    s = dense_setup
    M, T = s["M"], s["T"]
    V = lat.volume(s["L"])
    G5 = np.kron(np.eye(V), np.kron(D.gamma5(), np.eye(3)))
    Sfull = np.linalg.inv(M)
    Q1 = T.conj().T @ (G5 @ M) @ T
    S1 = T @ np.linalg.inv(Q1) @ T.conj().T @ G5
    D1 = T.conj().T @ M @ T
    assert rel(S1, T @ np.linalg.inv(D1) @ T.conj().T) < 1e-11
    S0 = Sfull - S1
    assert np.abs(T.conj().T @ M @ S0).max() < 1e-11 * np.abs(Sfull).max()
    assert np.abs(S0 @ M @ T).max() < 1e-11 * np.abs(Sfull).max()
    # the oracle's piecewise solve gives the same pieces
    eta = synthetic.z2_noise(s["L"], 1, 4)[0]
    psi, psi1, psi0 = S.pieces(s["U"], s["phi"], s["Dhat"], eta, s["kappa"], s["csw"], s["b"], tol=1e-12)
    e = eta.reshape(-1)
    assert rel(psi.reshape(-1), Sfull @ e) < 1e-10
    assert rel(psi1.reshape(-1), S1 @ e) < 1e-10
    assert rel(psi0.reshape(-1), S0 @ e) < 1e-9


@pytest.mark.parametrize("L,slab,bc", [((8, 2, 2, 2), 4, -1.0), ((7, 2, 2, 2), 3, -1.0), ((6, 2, 2, 2), 6, 1.0),
                                       ((3, 2, 2, 2), 1, -1.0)])
def test_slab_residual_equals_full_lattice(L, slab, bc):
    """The time-slab evaluation of D (one halo slice each side, boundary sign
    on the halo) reproduces the full-lattice D on every slice, including a
    ragged last slab, whole-lattice slabs and one-slice slabs, and the
    streamed residual equals the full one."""
    U = synthetic.gauge_links(L, 0.3, 91)
    kappa, csw = 0.124, 1.3
    x = synthetic.random_spinors(L, 1, 92)[0]
    b = synthetic.random_spinors(L, 1, 93)[0]
    full = D.dirac(U, x, kappa, csw, bc)
    for t0 in range(0, L[0], slab):
        t1 = min(L[0], t0 + slab)
        got = S.dirac_slab(U, x, kappa, csw, t0, t1, bc)
        assert np.abs(got - full[t0:t1]).max() < 1e-13
    assert S.residual_slabs(U, x, b, kappa, csw, bc, slab) == pytest.approx(
        S.true_residual(U, x, b, kappa, csw, bc), rel=1e-13)
