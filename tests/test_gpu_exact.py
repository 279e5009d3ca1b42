"""GPU parity of the exact coarsest-level estimator (Sec. "Exact estimator on
the coarsest grid", Eq. G_LL:exact; Eq. coarse:gamma) against the FP64 oracle:
the coarse gamma5 gamma_k matrices, the dense inverse of Q_c and the exact
correlator C(x0, y0) / G(t) on every level of a three-level chain, and the
LMA limit (one block covering the lattice, basis from exact low modes of Q)."""
import numpy as np
import pytest

import synthetic
from oracle import contract as K
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG

pytestmark = pytest.mark.gpu

L, B0, NV, KAPPA, CSW = (4, 4, 4, 4), (2, 2, 2, 2), 4, 0.124, 1.4
BLOCKS = [(2, 2, 1, 1), (1, 1, 2, 2)]


@pytest.fixture(scope="module")
def m():
    import paper_2412_06347_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def ctx(m):
    c = m.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def chain(m, ctx):
    U = synthetic.gauge_links(L, 0.3, 71)
    g = m.mglma_gauge_load(ctx, L, U, KAPPA, CSW)
    sub = m.mglma_subspace_build(ctx, g, B0, NV, 3, 72, m.MGLMA_FP64)
    C = [m.mglma_coarse_build(ctx, g, sub, m.MGLMA_FP32)]
    for b in BLOCKS:
        C.append(m.mglma_coarse_build_next(ctx, C[-1], b, m.MGLMA_FP32))
    Lbs = [lat.block_grid(L, B0)]
    for b in BLOCKS:
        Lbs.append(lat.block_grid(Lbs[-1], b))
    # the oracle on the GPU's own basis and stencils (exported in FP64)
    phi = np.zeros((lat.volume(Lbs[0]), 2, NV, lat.volume(B0), 4, 3), dtype=np.complex128)
    m.mglma_subspace_export(sub, phi)
    Dh = []
    for c, Lb in zip(C, Lbs):
        d = np.zeros((9, lat.volume(Lb), 2 * NV, 2 * NV), dtype=np.complex128)
        m.mglma_coarse_export(c, d)
        Dh.append(d)
    Gams = [[K.coarse_gamma5_gamma(phi, L, B0, k) for k in (1, 2, 3)]]
    for l, b in enumerate(BLOCKS):
        Gams.append([K.coarse_gamma_next(G, Lbs[l], b) for G in Gams[-1]])
    yield dict(U=U, g=g, sub=sub, C=C, Lbs=Lbs, Dh=Dh, Gams=Gams)
    for c in reversed(C):
        m.mglma_coarse_free(c)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_coarse_gamma_matrices(m, ctx, chain):
    for l in range(3):
        V = lat.volume(chain["Lbs"][l])
        for k in (1, 2, 3):
            out = np.zeros((L[0], V, 2 * NV, 2 * NV), dtype=np.complex128)
            m.mglma_coarse_gamma5_gamma(ctx, chain["C"][l], k, out)
            ref = chain["Gams"][l][k - 1]
            assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max(), (l, k)


def test_dense_inverse_and_exact_correlator(m, ctx, chain):
    for l in range(3):
        Lb = chain["Lbs"][l]
        n = lat.volume(Lb) * 2 * NV
        Qi = np.zeros((n, n), dtype=np.complex128)
        m.mglma_coarse_dense_inverse(ctx, chain["C"][l], Qi)
        g5 = np.tile(MG.coarse_gamma5(NV), lat.volume(Lb))
        Q = g5[:, None] * MG.dense_coarse(chain["Dh"][l], Lb)
        assert np.abs(Qi @ Q - np.eye(n)).max() < 1e-11, l
        C_ref, G_ref = K.exact_coarse_correlator(chain["Dh"][l], Lb, chain["Gams"][l], L)
        corr = np.zeros((L[0], L[0]), dtype=np.complex128)
        G = np.zeros(L[0], dtype=np.complex128)
        m.mglma_exact_correlator(ctx, chain["C"][l], corr, G)
        scale = np.abs(C_ref).max()
        assert np.abs(corr - C_ref).max() <= 1e-11 * scale, l
        assert np.abs(G - G_ref).max() <= 1e-11 * scale, l


def test_dense_inverse_at_scale(m, ctx):
    """n = 2048 (8^4 lattice, 2^4 blocks, Nv 4): Gauss-Jordan with partial
    pivoting against numpy's inverse of the same Q_c."""
    Lf = (8, 8, 8, 8)
    U = synthetic.gauge_links(Lf, 0.3, 1001)
    g = m.mglma_gauge_load(ctx, Lf, U, 0.12, 1.0)
    sub = m.mglma_subspace_build(ctx, g, (2, 2, 2, 2), 4, 5, 2001, m.MGLMA_FP64)
    c = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_FP64)
    Lb = lat.block_grid(Lf, (2, 2, 2, 2))
    d = np.zeros((9, lat.volume(Lb), 8, 8), dtype=np.complex128)
    m.mglma_coarse_export(c, d)
    n = lat.volume(Lb) * 8
    Qi = np.zeros((n, n), dtype=np.complex128)
    m.mglma_coarse_dense_inverse(ctx, c, Qi)
    g5 = np.tile(MG.coarse_gamma5(4), lat.volume(Lb))
    ref = np.linalg.inv(g5[:, None] * MG.dense_coarse(d, Lb))
    assert np.abs(Qi - ref).max() <= 1e-10 * np.abs(ref).max()
    m.mglma_coarse_free(c)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_lma_limit_exact_modes(m, ctx):
    """LMA limit: one block covering the whole lattice, basis loaded from the
    nv lowest exact eigenvectors of Q (chirality split, Eq. mg_basis).  The
    low eigenvalues mu_c of Q reappear in Q_c (App. spectra), so 1 / mu_c are
    eigenvalues of the GPU's dense Q_c^-1, and the exact correlator of this
    level equals the oracle's."""
    Lf, nv = (4, 2, 2, 4), 3
    U = synthetic.gauge_links(Lf, 0.3, 9)
    kappa, csw = 0.125, 1.9
    M = D.dense_dirac(U, kappa, csw)
    V = lat.volume(Lf)
    G5 = np.kron(np.eye(V), np.kron(D.gamma5(), np.eye(3)))
    w, v = np.linalg.eigh(G5 @ M)
    order = np.argsort(np.abs(w))[:nv]
    modes = np.ascontiguousarray(v[:, order].T.reshape((nv,) + Lf + (4, 3)))
    g = m.mglma_gauge_load(ctx, Lf, U, kappa, csw)
    sub = m.mglma_subspace_load(ctx, g, Lf, nv, modes, m.MGLMA_FP64)
    c = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_FP64)
    n = 2 * nv
    Qi = np.zeros((n, n), dtype=np.complex128)
    m.mglma_coarse_dense_inverse(ctx, c, Qi)
    ev = np.linalg.eigvals(Qi)
    for mu in w[order]:
        assert np.min(np.abs(ev - 1.0 / mu)) < 1e-10 * abs(1.0 / mu)
    phi = np.zeros((1, 2, nv, V, 4, 3), dtype=np.complex128)
    m.mglma_subspace_export(sub, phi)
    d = np.zeros((9, 1, n, n), dtype=np.complex128)
    m.mglma_coarse_export(c, d)
    C_ref, G_ref = K.exact_coarse_correlator(d, (1, 1, 1, 1), [K.coarse_gamma5_gamma(phi, Lf, Lf, k)
                                                                for k in (1, 2, 3)], Lf)
    corr = np.zeros((Lf[0], Lf[0]), dtype=np.complex128)
    m.mglma_exact_correlator(ctx, c, corr, None)
    assert np.abs(corr - C_ref).max() <= 1e-11 * np.abs(C_ref).max()
    m.mglma_coarse_free(c)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)
