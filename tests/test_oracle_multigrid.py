"""Pins of the oracle's block basis, R0/T0 and coarse operator: QR
factorisation, orthonormality and projector identities (Sec. 2, Sec. 3),
brute-force dense R0 D T0 (Sec. 2, Fig. A), gamma5-hermiticity of the coarse
operator and the eigenvalue alignment of App. spectra."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


@pytest.fixture(scope="module")
def mg44():
    """4^4 lattice, 2^4 blocks (L/b = 2 in every direction), Nv = 3."""
    L, b, nv = (4, 4, 4, 4), (2, 2, 2, 2), 3
    U = synthetic.gauge_links(L, 0.3, 21)
    starts = synthetic.gaussian_start_vectors(L, nv, 22)
    phi = MG.subspace(U, starts, 0.12, 1.0, b, 2)
    return dict(L=L, b=b, nv=nv, U=U, phi=phi, kappa=0.12, csw=1.0)


def test_mr_smoothing_reduces_residual(small_lattice):
    U, L = small_lattice["U"], small_lattice["L"]
    v = synthetic.gaussian_start_vectors(L, 1, 3)[0]
    A = D.clover_matrix(U, 0.12, 1.0)
    ratios = []
    for n in range(0, 6):
        w = MG.mr_smooth(U, v, 0.12, 1.0, n, A=A)
        ratios.append(np.linalg.norm(D.dirac(U, w, 0.12, 1.0, A=A)))
    assert all(ratios[i + 1] < ratios[i] for i in range(5))
    # one MR step is the exact minimiser of ||D(v + a r)|| over complex a
    r = -D.dirac(U, v, 0.12, 1.0, A=A)
    w1 = MG.mr_smooth(U, v, 0.12, 1.0, 1, A=A)
    base = np.linalg.norm(D.dirac(U, w1, 0.12, 1.0, A=A))
    for da in (1e-3, 1e-3j, -1e-3):
        assert np.linalg.norm(D.dirac(U, w1 + da * r, 0.12, 1.0, A=A)) > base


def test_gram_schmidt_equals_qr():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(5, 40)) + 1j * rng.normal(size=(5, 40))
    phi = MG.block_gram_schmidt(u)
    q, r = np.linalg.qr(u.T)
    ph = np.diag(r) / np.abs(np.diag(r))
    q = q * ph[None, :]  # make R's diagonal real positive
    assert rel(phi, q.T) < 1e-13
    bad = np.vstack([u[:2], u[0:1] * (1 + 2j)])
    with pytest.raises(MG.RankError):
        MG.block_gram_schmidt(bad)


def test_basis_orthonormal_and_chiral(mg44):
    phi, nv = mg44["phi"], mg44["nv"]
    V1, nB = phi.shape[0], phi.shape[3]
    flat = phi.reshape(V1, 2 * nv, nB * 12)
    gram = np.einsum("yik,yjk->yij", flat.conj(), flat)
    assert np.allclose(gram, np.eye(2 * nv)[None], atol=1e-14)
    assert np.allclose(phi[:, 0, :, :, 2:, :], 0) and np.allclose(phi[:, 1, :, :, :2, :], 0)


def test_restrict_prolong_identities(mg44):
    L, b, phi, nv = mg44["L"], mg44["b"], mg44["phi"], mg44["nv"]
    V1 = phi.shape[0]
    T = MG.dense_prolongator(phi, L, b)
    assert np.allclose(T.conj().T @ T, np.eye(V1 * 2 * nv), atol=1e-13)  # R T = 1
    psi = synthetic.random_spinors(L, 1, 31)[0]
    # R = T^dag
    assert rel(MG.restrict(phi, psi, L, b).reshape(-1), T.conj().T @ psi.reshape(-1)) < 1e-14
    # P = T R is a projector that commutes with gamma5
    P = lambda v: MG.prolong(phi, MG.restrict(phi, v, L, b), L, b)  # noqa: E731
    assert rel(P(P(psi)), P(psi)) < 1e-13
    assert rel(P(D.apply_gamma5(psi)), D.apply_gamma5(P(psi))) < 1e-13


def test_basis_spans_projected_block_fields(mg44):
    """u = P_alpha theta_B v_c lies in range T: P u = u."""
    L, b, phi, U, nv = mg44["L"], mg44["b"], mg44["phi"], mg44["U"], mg44["nv"]
    starts = synthetic.gaussian_start_vectors(L, nv, 22)
    v = MG.mr_smooth(U, starts[1], 0.12, 1.0, 2)
    bo = lat.block_of_site(L, b).reshape(L)
    u = np.where((bo == 5)[..., None, None], D._spin(D.chiral_projector(1), v), 0)
    Pu = MG.prolong(phi, MG.restrict(phi, u, L, b), L, b)
    assert rel(Pu, u) < 1e-12


def _check_stencil_equals_dense(U, phi, L, b, kappa, csw):
    Lb = lat.block_grid(L, b)
    Dhat = MG.coarse_operator(U, phi, kappa, csw, b)
    T = MG.dense_prolongator(phi, L, b)
    dense = T.conj().T @ D.dense_dirac(U, kappa, csw) @ T
    assert rel(MG.dense_coarse(Dhat, Lb), dense) < 1e-13
    return Dhat, dense


def test_coarse_operator_equals_dense_RDT_L_over_b_2(mg44):
    _check_stencil_equals_dense(mg44["U"], mg44["phi"], mg44["L"], mg44["b"], 0.12, 1.0)


def test_coarse_operator_equals_dense_whole_lattice_and_L_over_b_3():
    # 6x2x2x2 with 2^4 blocks: L/b = 3 in time, 1 (one block) in space
    L, b, nv = (6, 2, 2, 2), (2, 2, 2, 2), 2
    U = synthetic.gauge_links(L, 0.3, 41)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 42), 0.125, 1.7, b, 1)
    _check_stencil_equals_dense(U, phi, L, b, 0.125, 1.7)
    # LMA limit: one block covering the whole 2^4 lattice
    L, b = (2, 2, 2, 2), (2, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.3, 43)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, 3, 44), 0.125, 1.7, b, 1)
    _check_stencil_equals_dense(U, phi, L, b, 0.125, 1.7)


def test_coarse_gamma5_hermiticity_and_slot_symmetry(mg44):
    """App. chirality: ((gamma5)_1 D1)^dag = (gamma5)_1 D1, and stencil-wise
    Dhat_{-mu}(y + mu) = g5 Dhat_{+mu}(y)^dag g5."""
    L, b, phi, U, nv = mg44["L"], mg44["b"], mg44["phi"], mg44["U"], mg44["nv"]
    Lb = lat.block_grid(L, b)
    Dhat = MG.coarse_operator(U, phi, 0.12, 1.0, b)
    g5 = np.tile(MG.coarse_gamma5(nv), lat.volume(Lb))
    Qh = g5[:, None] * MG.dense_coarse(Dhat, Lb)
    assert np.allclose(Qh, Qh.conj().T, atol=1e-13)
    g = MG.coarse_gamma5(nv)
    nbr = lat.coarse_neighbour_table(Lb)
    for mu in range(4):
        for y in range(nbr.shape[0]):
            lhs = Dhat[mu + 4, nbr[y, mu]]
            rhs = g[:, None] * Dhat[mu, y].conj().T * g[None, :]
            assert np.allclose(lhs, rhs, atol=1e-13)
    assert np.allclose(g[:, None] * Dhat[8] - np.conj(np.swapaxes(g[:, None] * Dhat[8], -1, -2)), 0, atol=1e-13)


def test_coarse_apply_and_adjoint(mg44):
    L, b, phi, U, nv = mg44["L"], mg44["b"], mg44["phi"], mg44["U"], mg44["nv"]
    Lb = lat.block_grid(L, b)
    Dhat = MG.coarse_operator(U, phi, 0.12, 1.0, b)
    X = synthetic.random_coarse(lat.volume(Lb), 2 * nv, 2, 5)
    M = MG.dense_coarse(Dhat, Lb)
    assert rel(MG.coarse_apply(Dhat, X, Lb)[1].reshape(-1), M @ X[1].reshape(-1)) < 1e-14
    assert rel(MG.coarse_apply_dagger(Dhat, X, Lb)[0].reshape(-1), M.conj().T @ X[0].reshape(-1)) < 1e-14
    # the coarse operator applied to R psi equals R D T R psi
    psi = synthetic.random_spinors(L, 1, 8)[0]
    lhs = MG.coarse_apply(Dhat, MG.restrict(phi, psi, L, b), Lb)
    Ppsi = MG.prolong(phi, MG.restrict(phi, psi, L, b), L, b)
    rhs = MG.restrict(phi, D.dirac(U, Ppsi, 0.12, 1.0), L, b)
    assert rel(lhs, rhs) < 1e-13


def test_coarse_operator_gauge_invariant(mg44):
    """D1[U^g, g phi] = D1[U, phi]."""
    L, b, phi, U = mg44["L"], mg44["b"], mg44["phi"], mg44["U"]
    g = synthetic.random_su3(L, 1.0, 77)
    sites = lat.block_sites(L, b)
    gl = g.reshape(-1, 3, 3)[sites]  # (V1, nB, 3, 3)
    phig = np.einsum("ykij,yacksj->yacksi", gl, phi)
    D1 = MG.coarse_operator(U, phi, 0.12, 1.0, b)
    D2 = MG.coarse_operator(D.gauge_transform_links(U, g), phig, 0.12, 1.0, b)
    assert rel(D2, D1) < 1e-13


def test_nonzero_block_count():
    """Fig. A: (2d + 1) V_k (N_s N_c)^2 non-zeros when L/b >= 3."""
    L, b, nv = (6, 6, 3, 3), (2, 2, 1, 1), 2
    U = synthetic.gauge_links(L, 0.3, 51)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 52), 0.12, 1.0, b, 1)
    Lb = lat.block_grid(L, b)
    M = MG.dense_coarse(MG.coarse_operator(U, phi, 0.12, 1.0, b), Lb)
    V1 = lat.volume(Lb)
    assert np.count_nonzero(np.abs(M) > 1e-15) == 9 * V1 * (2 * nv) ** 2


def test_eigenvalue_alignment_with_exact_modes():
    """App. spectra: with the basis built from exact low modes of Q the lowest
    N_c eigenvalues of Q reappear in Q1 = (gamma5)_1 D1."""
    L, b, nv = (4, 2, 2, 2), (2, 2, 2, 2), 4
    U = synthetic.gauge_links(L, 0.4, 61)
    kappa, csw = 0.125, 1.5
    M = D.dense_dirac(U, kappa, csw)
    V = lat.volume(L)
    G5 = np.kron(np.eye(V), np.kron(D.gamma5(), np.eye(3)))
    w, v = np.linalg.eigh(G5 @ M)
    order = np.argsort(np.abs(w))[:nv]
    modes = v[:, order].T.reshape((nv,) + L + (4, 3))
    phi = MG.build_basis(modes, L, b)
    Lb = lat.block_grid(L, b)
    Dhat = MG.coarse_operator(U, phi, kappa, csw, b)
    g5 = np.tile(MG.coarse_gamma5(nv), lat.volume(Lb))
    wc = np.linalg.eigvalsh(g5[:, None] * MG.dense_coarse(Dhat, Lb))
    for lam in w[order]:
        assert np.min(np.abs(wc - lam)) < 1e-11


def test_cg_relaxation_filters_towards_low_modes():
    """CG on D^dag D x = 0 from a random start: ||D x|| / ||x|| falls with
    the step count and the iterate's weight moves onto the low modes of Q
    (App. chirality: the low right singular vectors of D are the low modes of Q)."""
    L = (4, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.3, 81)
    kappa, csw = 0.125, 1.0
    M = D.dense_dirac(U, kappa, csw)
    V = lat.volume(L)
    G5 = np.kron(np.eye(V), np.kron(D.gamma5(), np.eye(3)))
    w, v = np.linalg.eigh(G5 @ M)
    low = v[:, np.argsort(np.abs(w))[:12]]
    x0 = synthetic.gaussian_start_vectors(L, 1, 82)[0]
    frac, ratio = [], []
    for n in (0, 5, 20):
        x = MG.cg_relax(U, x0, kappa, csw, n).reshape(-1)
        frac.append(np.linalg.norm(low.conj().T @ x) / np.linalg.norm(x))
        ratio.append(np.linalg.norm(M @ x) / np.linalg.norm(x))
    assert ratio[0] > ratio[1] > ratio[2]
    assert frac[0] < frac[1] < frac[2] and frac[2] > 0.8
    # zero steps is the identity; the step is the CG minimiser along the first direction
    assert np.array_equal(MG.cg_relax(U, x0, kappa, csw, 0), x0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_cg_relaxation_is_the_krylov_minimiser(n):
    """CG on the normal equations D^dag D x = 0 from x0 is, after n steps, the
    unique minimiser of ||D x|| over x0 + K_n(D^dag D, D^dag D x0) -- the
    defining property of CG (it minimises the D^dag D-norm of the error, and
    the solution is 0).  The minimiser is computed independently: an
    orthonormal basis of the Krylov space from the dense D, then least
    squares.  A wrong step length, a wrong beta or a dropped direction gives
    another point of the affine space and fails."""
    L = (4, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.3, 83)
    kappa, csw = 0.125, 1.2
    M = D.dense_dirac(U, kappa, csw)
    x0 = synthetic.gaussian_start_vectors(L, 1, 84)[0].reshape(-1)
    N = M.conj().T @ M
    # Arnoldi (two Gram-Schmidt passes per vector) on N from N x0: an
    # orthonormal basis of K_n without the power basis's ill-conditioning
    Qk = np.empty((x0.size, n), dtype=np.complex128)
    v = N @ x0
    for j in range(n):
        for _ in range(2):
            v = v - Qk[:, :j] @ (Qk[:, :j].conj().T @ v)
        Qk[:, j] = v / np.linalg.norm(v)
        v = N @ Qk[:, j]
    c, *_ = np.linalg.lstsq(M @ Qk, -(M @ x0), rcond=None)
    x_min = x0 + Qk @ c
    x_cg = MG.cg_relax(U, x0.reshape(L + (4, 3)), kappa, csw, n).reshape(-1)
    assert np.linalg.norm(x_cg - x_min) / np.linalg.norm(x_min) < 1e-12
    # and it is a strict improvement on the previous step's minimiser
    if n > 1:
        x_prev = MG.cg_relax(U, x0.reshape(L + (4, 3)), kappa, csw, n - 1).reshape(-1)
        assert np.linalg.norm(M @ x_cg) < np.linalg.norm(M @ x_prev)
