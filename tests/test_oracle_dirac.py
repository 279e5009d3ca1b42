"""Pins of the oracle's lattice, gamma matrices and Dirac operator to facts
that do not come from the oracle: hand-computed index tables, the Clifford
algebra, the free-field momentum-space operator, an abelian constant field,
gamma5-hermiticity and gauge covariance."""
import itertools

import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


# ---------------------------------------------------------------- geometry
def test_neighbour_table_matches_brute_force():
    for L in [(4, 3, 2, 5), (2, 2, 2, 2), (3, 1, 4, 2)]:
        assert np.array_equal(lat.neighbour_table(L), lat.brute_force_neighbours(L))


def test_neighbour_table_hand_values():
    L = (4, 3, 2, 5)
    nb = lat.neighbour_table(L)
    # site 0 = (0,0,0,0): +t -> (1,0,0,0) = 30, -t -> (3,0,0,0) = 90,
    # +x1 -> (0,1,0,0) = 10, -x3 -> (0,0,0,4) = 4
    assert nb[0, 0] == 30 and nb[0, 4] == 90 and nb[0, 1] == 10 and nb[0, 7] == 4
    # last site (3,2,1,4) = 119: +t wraps to (0,2,1,4) = 29
    assert nb[119, 0] == 29


def test_block_maps_partition_the_lattice():
    L, b = (4, 4, 6, 2), (2, 2, 3, 1)
    sites = lat.block_sites(L, b)
    assert sites.shape == (2 * 2 * 2 * 2, 12)
    assert np.array_equal(np.sort(sites.ravel()), np.arange(lat.volume(L)))
    x = lat.coords(L)
    for y in range(sites.shape[0]):
        yy = x[sites[y]] // np.array(b)
        assert (yy == yy[0]).all()
    with pytest.raises(ValueError):
        lat.block_grid((4, 4, 4, 4), (3, 2, 2, 2))


# ------------------------------------------------------------ gamma algebra
def test_clifford_algebra_and_chiral_basis():
    g = D.gammas()
    for mu, nu in itertools.product(range(4), repeat=2):
        ac = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(ac, 2 * (mu == nu) * np.eye(4), atol=1e-15)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
    assert np.allclose(D.gamma5(), np.diag([1, 1, -1, -1]))
    assert np.allclose(D.chiral_projector(0), np.diag([1, 1, 0, 0]))
    assert np.allclose(D.chiral_projector(1), np.diag([0, 0, 1, 1]))
    # sigma_12 in this basis, worked out by hand: -(sigma_3 (+) sigma_3)
    assert np.allclose(D.sigma(1, 2), np.diag([-1, 1, -1, 1]))


# --------------------------------------------------------------- free field
def _plane_wave(L, p, u):
    x = lat.coords(L)
    phase = np.exp(1j * (x @ np.asarray(p))).reshape(tuple(L))
    return phase[..., None, None] * u


def _free_symbol(p, m0):
    g = D.gammas()
    M = (m0 + sum(1 - np.cos(pm) for pm in p)) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        M = M + 1j * np.sin(p[mu]) * g[mu]
    return M


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 2, 3, 4)])
def test_free_field_plane_waves(L):
    kappa = 0.13
    m0 = 1 / (2 * kappa) - 4
    U = synthetic.free_links(L)
    rng = np.random.default_rng(0)
    for n in [(0, 0, 0, 0), (1, 1, 2, 3), (L[0] - 1, 0, 1, 1)]:
        p = [(2 * n[0] + 1) * np.pi / L[0]] + [2 * np.pi * n[k] / L[k] for k in (1, 2, 3)]
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = _plane_wave(L, p, u)
        out = D.dirac(U, psi, kappa, 1.7)
        expect = _plane_wave(L, p, _free_symbol(p, m0) @ u)
        assert rel(out, expect) < 1e-13


def test_free_field_dense_spectrum():
    L = (4, 2, 2, 2)
    kappa = 0.125
    m0 = 1 / (2 * kappa) - 4
    M = D.dense_dirac(synthetic.free_links(L), kappa, 1.0)
    ev = np.linalg.eigvals(M)
    expect = []
    for n in itertools.product(*[range(v) for v in L]):
        p = [(2 * n[0] + 1) * np.pi / L[0]] + [2 * np.pi * n[k] / L[k] for k in (1, 2, 3)]
        a = m0 + sum(1 - np.cos(pm) for pm in p)
        s = np.sqrt(sum(np.sin(pm) ** 2 for pm in p))
        expect += [a + 1j * s] * 6 + [a - 1j * s] * 6
    expect = np.array(expect)
    assert np.allclose(np.sort(ev.real), np.sort(expect.real), atol=1e-12)
    assert np.allclose(np.sort(ev.imag), np.sort(expect.imag), atol=1e-12)
    # Q = gamma5 D is Hermitian with eigenvalues +-|D(p)|
    Q = np.kron(np.eye(len(expect) // 12), np.kron(D.gamma5(), np.eye(3))) @ M
    assert np.allclose(Q, Q.conj().T, atol=1e-14)
    assert np.allclose(np.sort(np.abs(np.linalg.eigvalsh(Q))), np.sort(np.abs(expect)), atol=1e-12)


# ----------------------------------------------------- abelian clover field
def test_abelian_constant_field_clover():
    L = (2, 4, 4, 2)
    phi = 2 * np.pi / (L[1] * L[2])
    csw, kappa = 1.7, 0.125
    U = synthetic.free_links(L)
    x = lat.coords(L).reshape(tuple(L) + (4,))
    for colour, q in ((0, 1.0), (1, -1.0)):
        U[..., 2, colour, colour] = np.exp(1j * q * phi * x[..., 1])
        edge = x[..., 1] == L[1] - 1
        U[..., 1, colour, colour] = np.where(edge, np.exp(-1j * q * phi * L[1] * x[..., 2]), 1.0)
    A = D.clover_matrix(U, kappa, csw)
    m0 = 1 / (2 * kappa) - 4
    C = A - (4 + m0) * np.einsum("st,ab->satb", np.eye(4), np.eye(3))
    s = 0.5 * csw * np.sin(phi)
    # by hand: colour 0 carries -(csw/2) sin(phi) sigma_12 = s diag(1,-1,1,-1);
    # colour 1 the opposite sign; colour 2 nothing; no colour mixing
    expect0 = s * np.diag([1, -1, 1, -1])
    assert np.allclose(C[..., :, 0, :, 0], expect0, atol=1e-14)
    assert np.allclose(C[..., :, 1, :, 1], -expect0, atol=1e-14)
    assert np.allclose(C[..., :, 2, :, 2], 0, atol=1e-14)
    assert np.allclose(C[..., :, 0, :, 1], 0, atol=1e-14)
    ev = np.linalg.eigvalsh(C[0, 0, 0, 0][:, 0, :, 0])
    assert np.allclose(ev, [-s, -s, s, s], atol=1e-14)


def test_clover_vanishes_on_pure_gauge():
    L = (4, 2, 2, 4)
    g = synthetic.random_su3(L, 0.7, 5)
    U = D.gauge_transform_links(synthetic.free_links(L), g)
    A = D.clover_matrix(U, 0.125, 1.9)
    assert np.allclose(A, 4.0 * np.einsum("st,ab->satb", np.eye(4), np.eye(3)), atol=1e-13)


# ------------------------------------------------------------ symmetries
def test_clover_hermitian_and_chirally_block_diagonal(small_lattice):
    A = D.clover_matrix(small_lattice["U"], 0.12, 1.0)
    M = A.reshape(A.shape[:4] + (12, 12))
    assert np.allclose(M, np.conj(np.swapaxes(M, -1, -2)), atol=1e-14)
    assert np.allclose(A[..., :2, :, 2:, :], 0, atol=1e-15)
    assert np.allclose(A[..., 2:, :, :2, :], 0, atol=1e-15)


def test_gamma5_hermiticity(small_lattice):
    U, k, c = small_lattice["U"], small_lattice["kappa"], small_lattice["csw"]
    L = small_lattice["L"]
    chi, psi = synthetic.random_spinors(L, 2, 3)
    lhs = np.vdot(chi, D.hermitian_dirac(U, psi, k, c))
    rhs = np.vdot(D.hermitian_dirac(U, chi, k, c), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    # and D^dag really is the adjoint of D
    lhs = np.vdot(chi, D.dirac(U, psi, k, c))
    rhs = np.vdot(D.dirac_dagger(U, chi, k, c), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_gauge_covariance(small_lattice):
    U, k, c, L = small_lattice["U"], 0.125, 1.9, small_lattice["L"]
    g = synthetic.random_su3(L, 1.0, 9)
    psi = synthetic.random_spinors(L, 1, 4)[0]
    lhs = D.dirac(D.gauge_transform_links(U, g), D.gauge_transform_spinor(psi, g), k, c)
    rhs = D.gauge_transform_spinor(D.dirac(U, psi, k, c), g)
    assert rel(lhs, rhs) < 1e-13


def test_periodic_bc_differs_only_on_boundary_hops(small_lattice):
    U, L = small_lattice["U"], small_lattice["L"]
    psi = synthetic.random_spinors(L, 1, 6)[0]
    a = D.dirac(U, psi, 0.12, 1.0, bc_t=-1.0)
    p = D.dirac(U, psi, 0.12, 1.0, bc_t=+1.0)
    diff = np.abs(a - p).reshape(L[0], -1).max(axis=1)
    assert diff[1:-1].max() == 0 and diff[0] > 0 and diff[-1] > 0


def test_dirac_at_sites_matches_full(small_lattice):
    U, L = small_lattice["U"], small_lattice["L"]
    psi = synthetic.random_spinors(L, 1, 7)[0]
    full = D.dirac(U, psi, 0.12, 1.0).reshape(-1, 4, 3)
    sites = [0, 5, 63, 64 * 3 + 17, 255]
    assert rel(D.dirac_at_sites(U, psi, 0.12, 1.0, sites), full[sites]) < 1e-14
