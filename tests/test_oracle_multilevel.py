"""Pins of the oracle's inner levels (Sec. "Multigrid decompositions"):
R_l / T_l with the sqrt(V_{l+1} / V_l) factor, the recursive operator
D_{l+1} = R_l D_l T_l as a nine-slot stencil, and the pieces of the
telescoping decomposition, against dense matrices built from the fine
Wilson-clover operator on a 4^4 lattice."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG

# 4^4 fine lattice, 2^4 blocks -> level 1 on 2^4 (V1 16), then blocks of
# (2, 2, 1, 1) level-1 sites -> level 2 on 1x1x2x2 (V2 4), then (1, 1, 2, 2)
# -> level 3 with one site (the LMA limit of the hierarchy)
L, B0, NV = (4, 4, 4, 4), (2, 2, 2, 2), 2
BLOCKS = [(2, 2, 1, 1), (1, 1, 2, 2)]
KAPPA, CSW = 0.124, 1.4


@pytest.fixture(scope="module")
def hier():
    U = synthetic.gauge_links(L, 0.3, 61)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, NV, 62), KAPPA, CSW, B0, 3)
    Lbs = [lat.block_grid(L, B0)]
    Dh = [MG.coarse_operator(U, phi, KAPPA, CSW, B0)]
    for b in BLOCKS:
        Dh.append(MG.coarse_operator_next(Dh[-1], Lbs[-1], b))
        Lbs.append(lat.block_grid(Lbs[-1], b))
    M = D.dense_dirac(U, KAPPA, CSW)
    T0 = MG.dense_prolongator(phi, L, B0)
    return dict(U=U, phi=phi, Lbs=Lbs, Dh=Dh, M=M, T0=T0)


def dense_R(l, Lbs):
    """kron(R_l, 1_n) for the transfer from level l (l >= 1) to l + 1."""
    return np.kron(MG.dense_restrict_level(Lbs[l - 1], BLOCKS[l - 1]), np.eye(2 * NV))


def test_transfer_normalisation_and_adjoint(hier):
    """R_l T_l = 1 on the next level (the sqrt(V_{l+1}/V_l) factor), T_l =
    R_l^dag, and T_l R_l is an orthogonal projector."""
    rng = np.random.default_rng(5)
    for l in (1, 2):
        Lb, b = hier["Lbs"][l - 1], BLOCKS[l - 1]
        Lb2 = lat.block_grid(Lb, b)
        Y = rng.standard_normal((lat.volume(Lb2), 2 * NV)) + 1j * rng.standard_normal((lat.volume(Lb2), 2 * NV))
        assert np.allclose(MG.restrict_level(MG.prolong_level(Y, Lb, b), Lb, b), Y, atol=1e-14)
        X = rng.standard_normal((lat.volume(Lb), 2 * NV)) + 1j * rng.standard_normal((lat.volume(Lb), 2 * NV))
        lhs = np.vdot(Y, MG.restrict_level(X, Lb, b))
        rhs = np.vdot(MG.prolong_level(Y, Lb, b), X)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
        R = MG.dense_restrict_level(Lb, b)
        P = R.T @ R
        assert np.allclose(P @ P, P, atol=1e-14)
        # each row of R has |B| entries sqrt(V_{l+1}/V_l) = 1/sqrt(|B|)
        nb = int(np.prod(b))
        assert np.allclose(R[R != 0], 1.0 / np.sqrt(nb))


def test_recursive_operator_is_galerkin(hier):
    """The stencil D_{l+1} (slot-wise assembly) equals the dense R_l D_l T_l,
    and also the compound Galerkin product calR_l D calT_l from the fine
    operator -- on every level down to the one-site (LMA) grid."""
    Lbs, Dh, M, T0 = hier["Lbs"], hier["Dh"], hier["M"], hier["T0"]
    Tc = T0
    for l in (1, 2):
        dense_l = MG.dense_coarse(Dh[l - 1], Lbs[l - 1])
        R = dense_R(l, Lbs)
        dense_next = MG.dense_coarse(Dh[l], Lbs[l])
        assert np.abs(dense_next - R @ dense_l @ R.T).max() < 1e-13 * np.abs(dense_l).max()
        Tc = Tc @ R.T  # calT_{l+1} = T_0 ... T_l
        assert np.abs(dense_next - Tc.conj().T @ M @ Tc).max() < 1e-12 * np.abs(M).max()
    assert lat.volume(Lbs[-1]) == 1


def test_recursive_operator_gamma5_hermiticity(hier):
    """Q_{l+1} = g5hat D_{l+1} stays Hermitian on every level (the chirality
    split survives the aggregation, App. chirality)."""
    for l in range(3):
        Lb = hier["Lbs"][l]
        g5 = np.tile(MG.coarse_gamma5(NV), lat.volume(Lb))
        Q = g5[:, None] * MG.dense_coarse(hier["Dh"][l], Lb)
        assert np.abs(Q - Q.conj().T).max() < 1e-13 * np.abs(Q).max()


def test_pieces_galerkin_and_dense(hier):
    """psi_l = calT_l D_l^-1 calR_l eta equals the dense form, and the sum of
    the outer pieces S_0 + ... + S_{l-1} = D^-1 - calT_l D_l^-1 calR_l is
    Galerkin-orthogonal: calR_l D (x - psi_l) = 0 on every level."""
    U, phi, Lbs, Dh, M, T0 = (hier[k] for k in ("U", "phi", "Lbs", "Dh", "M", "T0"))
    eta = synthetic.z2_noise(L, 1, 63)[0]
    psis = MG.multilevel_pieces(Dh, Lbs, BLOCKS, phi, L, B0, eta, tol=1e-14)
    x = np.linalg.solve(M, eta.reshape(-1))
    Tc = T0
    for l in range(3):
        if l:
            Tc = Tc @ dense_R(l, Lbs).T
        Dl = Tc.conj().T @ M @ Tc
        ref = Tc @ np.linalg.solve(Dl, Tc.conj().T @ eta.reshape(-1))
        assert np.linalg.norm(psis[l].reshape(-1) - ref) < 1e-10 * np.linalg.norm(ref)
        g = Tc.conj().T @ (M @ (x - psis[l].reshape(-1)))
        assert np.linalg.norm(g) < 1e-10 * np.linalg.norm(eta)
    # the telescoping sum of the pieces gives back x = D^-1 eta
    S = [x - psis[0].reshape(-1)] + [(psis[l] - psis[l + 1]).reshape(-1) for l in range(2)] + [psis[2].reshape(-1)]
    assert np.linalg.norm(sum(S) - x) < 1e-13 * np.linalg.norm(x)


def test_recursive_operator_slots_on_a_long_grid():
    """A geometry whose level-2 grid has extent 3 in a blocked direction
    (12 x 2^3 fine sites, 2^4 blocks -> level 1 on 6 x 1^3, blocks of 2 ->
    level 2 on 3 x 1^3): a hop that stays inside its block must land in the
    self slot, one that leaves in the neighbour's, or the dense matrix of the
    stencil differs from R_1 D_1 T_1 and from calR_2 D calT_2."""
    Lf, b0, nv = (12, 2, 2, 2), (2, 2, 2, 2), 2
    U = synthetic.gauge_links(Lf, 0.3, 64)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(Lf, nv, 65), KAPPA, CSW, b0, 3)
    Lb1 = lat.block_grid(Lf, b0)
    D1 = MG.coarse_operator(U, phi, KAPPA, CSW, b0)
    b1 = (2, 1, 1, 1)
    D2 = MG.coarse_operator_next(D1, Lb1, b1)
    Lb2 = lat.block_grid(Lb1, b1)
    assert Lb2 == (3, 1, 1, 1)
    R = np.kron(MG.dense_restrict_level(Lb1, b1), np.eye(2 * nv))
    d2 = MG.dense_coarse(D2, Lb2)
    assert np.abs(d2 - R @ MG.dense_coarse(D1, Lb1) @ R.T).max() < 1e-13 * np.abs(d2).max()
    Tc = MG.dense_prolongator(phi, Lf, b0) @ R.T
    M = D.dense_dirac(U, KAPPA, CSW)
    assert np.abs(d2 - Tc.conj().T @ M @ Tc).max() < 1e-12 * np.abs(M).max()
    # the time-direction hops of level 2 are non-zero and live in their own slots
    assert np.abs(D2[0]).max() > 1e-3 and np.abs(D2[4]).max() > 1e-3
