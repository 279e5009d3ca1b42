"""Pins of the oracle's even-odd (Schur) decomposition, for the fine
Wilson-clover operator and the coarse stencil: every hop joins opposite
parities (the diagonal parity blocks are site-local), the Schur solve with
back-substitution reproduces the dense inverse, the determinant factorises
det M = det M_oo det S_ee (the block-LU identity), and g5 S_ee is Hermitian
(gamma5-hermiticity survives the Schur complement because the site-local
blocks commute with gamma5)."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG
from oracle import solvers as S


@pytest.fixture(scope="module")
def fine():
    L = (4, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.3, 91)
    M = D.dense_dirac(U, 0.124, 1.3)
    V = lat.volume(L)
    g5 = np.kron(np.eye(V), np.kron(D.gamma5(), np.eye(3)))
    return dict(L=L, M=M, par=S.parity(L), g5=g5, ndof=12)


@pytest.fixture(scope="module")
def coarse():
    L, b, nv = (4, 4, 4, 4), (2, 2, 2, 2), 2
    U = synthetic.gauge_links(L, 0.3, 92)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 93), 0.124, 1.3, b, 3)
    Lb = lat.block_grid(L, b)
    Dh = MG.coarse_operator(U, phi, 0.124, 1.3, b)
    M = MG.dense_coarse(Dh, Lb)
    g5 = np.diag(np.tile(MG.coarse_gamma5(nv), lat.volume(Lb)))
    return dict(L=Lb, M=M, par=S.parity(Lb), g5=g5, ndof=2 * nv)


@pytest.mark.parametrize("which", ["fine", "coarse"])
def test_parity_blocks(which, request):
    s = request.getfixturevalue(which)
    Mee, Meo, Moe, Moo = S.eo_blocks(s["M"], s["par"], s["ndof"])
    n = s["ndof"]
    for blk in (Mee, Moo):  # site-local: block-diagonal in sites
        for i in range(blk.shape[0] // n):
            for j in range(blk.shape[0] // n):
                if i != j:
                    assert np.abs(blk[i * n:(i + 1) * n, j * n:(j + 1) * n]).max() == 0
    assert np.abs(Meo).max() > 0 and np.abs(Moe).max() > 0


@pytest.mark.parametrize("which", ["fine", "coarse"])
def test_schur_solve_and_determinant(which, request):
    s = request.getfixturevalue(which)
    M, par, n = s["M"], s["par"], s["ndof"]
    b = np.random.default_rng(3).standard_normal(M.shape[0]) + 0j
    x = S.solve_eo(M, par, n, b)
    assert np.linalg.norm(x - np.linalg.solve(M, b)) < 1e-12 * np.linalg.norm(x)
    Se = S.schur_even(M, par, n)
    _, _, _, Moo = S.eo_blocks(M, par, n)
    s1, l1 = np.linalg.slogdet(M)
    s2, l2 = np.linalg.slogdet(Moo)
    s3, l3 = np.linalg.slogdet(Se)
    assert abs(l1 - (l2 + l3)) < 1e-10 * abs(l1) and abs(s1 - s2 * s3) < 1e-10


@pytest.mark.parametrize("which", ["fine", "coarse"])
def test_schur_gamma5_hermiticity(which, request):
    s = request.getfixturevalue(which)
    e = np.repeat(s["par"] == 0, s["ndof"])
    Q = s["g5"][np.ix_(e, e)] @ S.schur_even(s["M"], s["par"], s["ndof"])
    assert np.abs(Q - Q.conj().T).max() < 1e-12 * np.abs(Q).max()
