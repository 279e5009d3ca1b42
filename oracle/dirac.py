"""O(a)-improved Wilson-clover Dirac operator (oracle; test infrastructure only).

The paper works with N_f = 2 non-perturbatively O(a)-improved Wilson fermions
(Tab. ensembles: hopping parameter kappa and clover coefficient c_sw) and
defines Q = gamma5 D (Sec. 2).  It never prints D itself; the reading used
here is the standard Wilson-clover operator in the mass normalisation
m0 = 1/(2 kappa) - 4:

    (D psi)(x) = A(x) psi(x)
                 - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]
    A(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x)
    sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]
    Fhat_{mu nu}(x) = (1/8) [Q_{mu nu}(x) - Q_{nu mu}(x)]

with Q_{mu nu}(x) the sum of the four plaquettes of the mu-nu plane that start
and end at x, each run mu-then-nu (the clover leaves).  Gauge links are
periodic; a fermion hop that crosses the time boundary x0 = L0-1 <-> 0 is
multiplied by ``bc_t`` (-1: antiperiodic).

Gamma matrices: the chiral basis, in 2x2 blocks
gamma0 = [[0, -1], [-1, 0]], gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
so gamma5 = gamma0 gamma1 gamma2 gamma3 = diag(1, 1, -1, -1) and the chiral
projectors P_alpha = (1 + (-1)^alpha gamma5)/2 of Eq. mg_basis select spins
{0, 1} (alpha = 0) and {2, 3} (alpha = 1).

Arrays: a spinor field is (L0, L1, L2, L3, 4, 3) complex128, a batch puts a
leading RHS axis in front; links are (L0, L1, L2, L3, 4, 3, 3).
"""
from __future__ import annotations

import numpy as np

_PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def gammas() -> np.ndarray:
    """gamma_0 .. gamma_3 in the chiral basis, shape (4, 4, 4)."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    eye = np.eye(2)
    g[0][:2, 2:] = -eye
    g[0][2:, :2] = -eye
    for k in range(3):
        g[k + 1][:2, 2:] = -1j * _PAULI[k]
        g[k + 1][2:, :2] = 1j * _PAULI[k]
    return g


def gamma5() -> np.ndarray:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigma(mu: int, nu: int) -> np.ndarray:
    g = gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def chiral_projector(alpha: int) -> np.ndarray:
    """P_alpha = (1 + (-1)^alpha gamma5) / 2 (Eq. mg_basis)."""
    return 0.5 * (np.eye(4) + (-1) ** alpha * gamma5())


def m0_from_kappa(kappa: float) -> float:
    return 1.0 / (2.0 * kappa) - 4.0


def shift(f: np.ndarray, mu: int, step: int) -> np.ndarray:
    """g(x) = f(x + step * mu_hat), periodic; axis mu of ``f`` is direction mu."""
    return np.roll(f, -step, axis=mu)


def dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_{mu nu}(x): the four mu-nu plaquettes that start and end at x, each
    traversed in the rotation sense +mu -> +nu -> -mu -> -nu."""
    Um = U[..., mu, :, :]
    Un = U[..., nu, :, :]
    s = shift
    l1 = Um @ s(Un, mu, 1) @ dag(s(Um, nu, 1)) @ dag(Un)
    l2 = Un @ dag(s(s(Um, nu, 1), mu, -1)) @ dag(s(Un, mu, -1)) @ s(Um, mu, -1)
    l3 = dag(s(Um, mu, -1)) @ dag(s(s(Un, mu, -1), nu, -1)) @ s(s(Um, mu, -1), nu, -1) @ s(Un, nu, -1)
    l4 = dag(s(Un, nu, -1)) @ s(Um, nu, -1) @ s(s(Un, nu, -1), mu, 1) @ dag(Um)
    return l1 + l2 + l3 + l4


def field_strength(U: np.ndarray) -> dict:
    """Fhat_{mu nu}(x) = (Q_{mu nu} - Q_{nu mu}) / 8 for every ordered pair
    mu != nu, each Q evaluated from its own leaves."""
    F = {}
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                F[(mu, nu)] = (leaves(U, mu, nu) - leaves(U, nu, mu)) / 8.0
    return F


def clover_matrix(U: np.ndarray, kappa: float, csw: float) -> np.ndarray:
    """A(x) = (4 + m0) 1 + c_sw (i/4) sum_{mu != nu} sigma_{mu nu} (x) Fhat_{mu nu}(x),
    shape (L0, L1, L2, L3, 4, 3, 4, 3) with index order [spin, colour, spin', colour']."""
    lat = U.shape[:4]
    m0 = m0_from_kappa(kappa)
    A = np.zeros(lat + (4, 3, 4, 3), dtype=np.complex128)
    eye = np.einsum("st,ab->satb", np.eye(4), np.eye(3))
    A += (4.0 + m0) * eye
    F = field_strength(U)
    for (mu, nu), f in F.items():
        A += csw * 0.25j * np.einsum("st,...ab->...satb", sigma(mu, nu), f)
    return A


def apply_clover(A: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return np.einsum("...satb,...tb->...sa", A, psi)


def _colour(U3: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)[s, a] = sum_b U[a, b] psi[s, b] at every site."""
    return np.swapaxes(U3 @ np.swapaxes(psi, -1, -2), -1, -2)


def _spin(G: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return np.einsum("st,...tc->...sc", G, psi)


def _boundary_sign(lat, mu: int, forward: bool, bc_t: float) -> np.ndarray:
    """Sign of the hop leaving each site in direction +mu (forward) or -mu:
    bc_t where the hop crosses the time boundary, 1 elsewhere."""
    s = np.ones(lat, dtype=np.float64)
    if mu == 0:
        if forward:
            s[lat[0] - 1] = bc_t
        else:
            s[0] = bc_t
    return s[..., None, None]


def hop(U: np.ndarray, psi: np.ndarray, d: int, bc_t: float = -1.0) -> np.ndarray:
    """One hopping term of D for hop slot d (single field):
    d = mu < 4:  -1/2 (1 - gamma_mu) U_mu(x) psi(x + mu)
    d = mu + 4:  -1/2 (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
    including the time-boundary sign."""
    lat = psi.shape[:4]
    g = gammas()
    one = np.eye(4)
    if d < 4:
        mu = d
        v = _colour(U[..., mu, :, :], shift(psi, mu, 1))
        v = _spin(one - g[mu], v)
        return -0.5 * _boundary_sign(lat, mu, True, bc_t) * v
    mu = d - 4
    v = _colour(dag(shift(U[..., mu, :, :], mu, -1)), shift(psi, mu, -1))
    v = _spin(one + g[mu], v)
    return -0.5 * _boundary_sign(lat, mu, False, bc_t) * v


def dirac(U, psi, kappa, csw, bc_t=-1.0, A=None) -> np.ndarray:
    """D psi for one field (L..., 4, 3) or a batch (n, L..., 4, 3)."""
    if psi.ndim == 7:
        return np.stack([dirac(U, p, kappa, csw, bc_t, A) for p in psi])
    if A is None:
        A = clover_matrix(U, kappa, csw)
    out = apply_clover(A, psi)
    for d in range(8):
        out += hop(U, psi, d, bc_t)
    return out


def apply_gamma5(psi: np.ndarray) -> np.ndarray:
    return _spin(gamma5(), psi)


def dirac_dagger(U, psi, kappa, csw, bc_t=-1.0, A=None) -> np.ndarray:
    """D^dag = gamma5 D gamma5 (gamma5-hermiticity of the Wilson-clover D)."""
    return apply_gamma5(dirac(U, apply_gamma5(psi), kappa, csw, bc_t, A))


def hermitian_dirac(U, psi, kappa, csw, bc_t=-1.0, A=None) -> np.ndarray:
    """Q psi = gamma5 D psi (Sec. 2)."""
    return apply_gamma5(dirac(U, psi, kappa, csw, bc_t, A))


def dense_dirac(U, kappa, csw, bc_t=-1.0) -> np.ndarray:
    """The (12V x 12V) matrix of D, column j = D e_j (small lattices only)."""
    lat = U.shape[:4]
    n = int(np.prod(lat)) * 12
    A = clover_matrix(U, kappa, csw)
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = dirac(U, e.reshape(lat + (4, 3)), kappa, csw, bc_t, A).reshape(-1)
    return M


def gauge_transform_links(U, g) -> np.ndarray:
    """U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dag."""
    out = np.empty_like(U)
    for mu in range(4):
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ dag(shift(g, mu, 1))
    return out


def gauge_transform_spinor(psi, g) -> np.ndarray:
    return _colour(g, psi)


def dirac_at_sites(U, psi, kappa, csw, sites, bc_t=-1.0) -> np.ndarray:
    """(D psi)(x) at a short list of flat site indices, evaluated site by site
    from the definition (only the links and spinors around each site are
    touched), for spot checks on lattices too large for ``dirac``.  Returns
    (len(sites), 4, 3)."""
    lat = [int(v) for v in psi.shape[:4]]
    g = gammas()
    one = np.eye(4)
    m0 = m0_from_kappa(kappa)
    out = np.zeros((len(sites), 4, 3), dtype=np.complex128)

    def at(x):
        return tuple(int(x[m]) % lat[m] for m in range(4))

    def Ul(x, mu):
        return U[at(x) + (mu,)]

    def plaq_sum(x, mu, nu):
        e = np.eye(4, dtype=np.int64)
        xm = np.asarray(x)
        D = lambda M: np.conj(M.T)  # noqa: E731
        l1 = Ul(xm, mu) @ Ul(xm + e[mu], nu) @ D(Ul(xm + e[nu], mu)) @ D(Ul(xm, nu))
        l2 = Ul(xm, nu) @ D(Ul(xm + e[nu] - e[mu], mu)) @ D(Ul(xm - e[mu], nu)) @ Ul(xm - e[mu], mu)
        l3 = D(Ul(xm - e[mu], mu)) @ D(Ul(xm - e[mu] - e[nu], nu)) @ Ul(xm - e[mu] - e[nu], mu) @ Ul(xm - e[nu], nu)
        l4 = D(Ul(xm - e[nu], nu)) @ Ul(xm - e[nu], mu) @ Ul(xm - e[nu] + e[mu], nu) @ D(Ul(xm, mu))
        return l1 + l2 + l3 + l4

    for n, s in enumerate(sites):
        s = int(s)
        x = [0, 0, 0, 0]
        r = s
        for m in (3, 2, 1, 0):
            x[m] = r % lat[m]
            r //= lat[m]
        xm = np.asarray(x, dtype=np.int64)
        e = np.eye(4, dtype=np.int64)
        A = (4.0 + m0) * np.einsum("st,ab->satb", np.eye(4), np.eye(3)).astype(np.complex128)
        for mu in range(4):
            for nu in range(4):
                if mu != nu:
                    F = (plaq_sum(xm, mu, nu) - plaq_sum(xm, nu, mu)) / 8.0
                    A += csw * 0.25j * np.einsum("st,ab->satb", sigma(mu, nu), F)
        acc = np.einsum("satb,tb->sa", A, psi[at(xm)])
        for mu in range(4):
            sf = bc_t if (mu == 0 and x[0] == lat[0] - 1) else 1.0
            sb = bc_t if (mu == 0 and x[0] == 0) else 1.0
            v = (Ul(xm, mu) @ psi[at(xm + e[mu])].T).T
            acc += -0.5 * sf * ((one - g[mu]) @ v)
            w = (np.conj(Ul(xm - e[mu], mu).T) @ psi[at(xm - e[mu])].T).T
            acc += -0.5 * sb * ((one + g[mu]) @ w)
        out[n] = acc
    return out
