"""Block basis, restrictor, prolongator and coarse operator (oracle; test
infrastructure only).

* Test vectors.  The paper builds its basis from exact low modes of Q
  (Sec. 3) and states that inexact modes work the same way (Sec. 3, opening
  paragraphs; Sec. conclusion).  The reading used here: N_v random starts, each
  relaxed by ``n_smooth`` minimal-residual steps on D v = 0
  (r = -D v; alpha = <D r, r> / <D r, D r>; v += alpha r; r -= alpha D r),
  optionally followed by ``n_cg`` CG steps on the normal equations of
  D x = 0 (``cg_relax``), which filter towards the low modes of Q.
* Chirality-split block fields (Eq. mg_basis): u_{alpha c}^{B_y} =
  P_alpha theta_{B_y} v_c, orthonormalised inside each block and chirality by
  Gram-Schmidt (modified Gram-Schmidt, two passes, then normalisation; a
  vector whose remaining norm is <= 1e-12 of its starting norm is rank
  deficient and raises).
* R0 (Eq. res_mg): (R psi)_{alpha c}(y) = sum_{x in B_y} phi_{alpha c}^{B_y}(x)^dag psi(x).
* T0 (Eq. pro_mg): (T psi1)(x) = sum_{alpha c} psi1_{alpha c}(y(x)) phi_{alpha c}^{B_y}(x).
* Coarse operator D1 = R0 D T0 (Sec. 2 with Q replaced by D, equivalent by
  App. chirality since [P, gamma5] = 0), stored as the nine-slot stencil of
  Fig. A: Dhat[d, y] maps X(nbr_d(y)) into Y(y).  Slot d < 8 collects the
  hopping terms of D that cross the face of B_y in hop direction d (the
  neighbour block may be y itself when L_mu / b_mu = 1, and the +mu and -mu
  neighbours coincide when L_mu / b_mu = 2; slots stay separate and are summed
  on application); slot 8 collects the clover term and every hop that stays
  inside B_y.

* Inner levels (Sec. "Multigrid decompositions"): for l >= 1 the restrictor
  R_l of a coarse field psi_l on the grid Lambda_l sums the components of
  equal (alpha, c) over the level-l sites z whose block of the next level is
  y, times sqrt(V_{l+1} / V_l); the prolongator T_l copies psi_{l+1}(y) to
  every such z with the same factor.  The coarse operator of the next level
  is Q_{l+1} = R_l Q_l T_l; with Q_l = g5hat D_l and R_l acting per (alpha, c)
  this is g5hat D_{l+1}, D_{l+1} = R_l D_l T_l, again a nine-slot stencil:
  slot d < 8 of y collects the slot-d blocks of the sites z of B_y whose
  slot-d neighbour lies outside B_y, slot 8 the self blocks and every block
  whose neighbour stays inside, all times V_{l+1} / V_l.

Arrays: the basis is phi[y, alpha, c, k, spin, colour] over the |B| sites k of
block y (site-in-block order) with the spins of the other chirality zero;
coarse fields are (V1, 2 N_v) with dof index alpha*N_v + c; a coarse batch
puts the RHS axis first.
"""
from __future__ import annotations

import numpy as np

from . import dirac as _d
from . import lattice as _lat


class RankError(ValueError):
    """Raised when a block basis vector is linearly dependent on earlier ones."""


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def mr_smooth(U, v, kappa, csw, n_smooth, bc_t=-1.0, A=None) -> np.ndarray:
    """n_smooth minimal-residual steps on D v = 0 for one field."""
    if A is None:
        A = _d.clover_matrix(U, kappa, csw)
    v = v.copy()
    r = -_d.dirac(U, v, kappa, csw, bc_t, A)
    for _ in range(n_smooth):
        w = _d.dirac(U, r, kappa, csw, bc_t, A)
        alpha = inner(w, r) / inner(w, w).real
        v += alpha * r
        r -= alpha * w
    return v


def cg_relax(U, v, kappa, csw, n_cg, bc_t=-1.0, A=None) -> np.ndarray:
    """n_cg conjugate-gradient steps on the normal equations of D x = 0 from
    x0 = v (one field): the iterate minimises ||D x|| over x0 + Krylov space,
    so it keeps mostly the low right singular vectors of D, which App.
    chirality identifies with the low modes of Q.  Fixed step count, no
    stopping test."""
    if A is None:
        A = _d.clover_matrix(U, kappa, csw)
    x = v.copy()
    r = -_d.dirac(U, x, kappa, csw, bc_t, A)
    z = _d.dirac_dagger(U, r, kappa, csw, bc_t, A)
    p = z.copy()
    zz = inner(z, z).real
    for _ in range(n_cg):
        w = _d.dirac(U, p, kappa, csw, bc_t, A)
        a = zz / inner(w, w).real
        x += a * p
        r -= a * w
        z = _d.dirac_dagger(U, r, kappa, csw, bc_t, A)
        zz_new = inner(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
    return x


def block_gram_schmidt(u: np.ndarray) -> np.ndarray:
    """Orthonormalise the rows u[c] (vectors) in order c = 0, 1, ...:
    two passes of modified Gram-Schmidt against the finished phi_j, j < c,
    then normalisation."""
    n = u.shape[0]
    phi = np.zeros_like(u)
    for c in range(n):
        w = u[c].copy()
        start = np.linalg.norm(w)
        for _ in range(2):
            for j in range(c):
                w -= np.vdot(phi[j], w) * phi[j]
        nrm = np.linalg.norm(w)
        if not nrm > 1e-12 * start:
            raise RankError(f"basis vector {c} is rank deficient ({nrm:.3e} of {start:.3e})")
        phi[c] = w / nrm
    return phi


def build_basis(vecs: np.ndarray, L, b) -> np.ndarray:
    """phi[y, alpha, c, k, s, a] from test vectors vecs (Nv, L..., 4, 3):
    P_alpha theta_{B_y} v_c, then Gram-Schmidt per (block, chirality)."""
    nv = vecs.shape[0]
    sites = _lat.block_sites(L, b)  # (V1, nB)
    V1, nB = sites.shape
    flat = vecs.reshape(nv, -1, 4, 3)
    phi = np.zeros((V1, 2, nv, nB, 4, 3), dtype=np.complex128)
    for alpha in range(2):
        P = _d.chiral_projector(alpha)
        proj = np.einsum("st,nvtc->nvsc", P, flat)
        for y in range(V1):
            u = proj[:, sites[y]]  # (nv, nB, 4, 3)
            phi[y, alpha] = block_gram_schmidt(u.reshape(nv, -1)).reshape(nv, nB, 4, 3)
    return phi


def make_test_vectors(U, starts, kappa, csw, n_smooth, n_cg=0, bc_t=-1.0) -> np.ndarray:
    """Random starts -> n_smooth MR steps -> n_cg CG steps on D x = 0."""
    A = _d.clover_matrix(U, kappa, csw)
    out = []
    for s in starts:
        v = mr_smooth(U, s, kappa, csw, n_smooth, bc_t, A)
        if n_cg:
            v = cg_relax(U, v, kappa, csw, n_cg, bc_t, A)
        out.append(v)
    return np.stack(out)


def subspace(U, starts, kappa, csw, b, n_smooth, bc_t=-1.0, n_cg=0) -> np.ndarray:
    """Test vectors from random starts (smoothing, relaxation), then the block
    basis."""
    vecs = make_test_vectors(U, starts, kappa, csw, n_smooth, n_cg, bc_t)
    return build_basis(vecs, U.shape[:4], b)


def restrict(phi: np.ndarray, psi: np.ndarray, L, b) -> np.ndarray:
    """R0 psi (Eq. res_mg) for one field -> (V1, 2 Nv), or a batch."""
    if psi.ndim == 7:
        return np.stack([restrict(phi, p, L, b) for p in psi])
    sites = _lat.block_sites(L, b)
    V1, _, nv = phi.shape[:3]
    loc = psi.reshape(-1, 4, 3)[sites]  # (V1, nB, 4, 3)
    out = np.einsum("yacksi,yksi->yac", np.conj(phi), loc)
    return out.reshape(V1, 2 * nv)


def prolong(phi: np.ndarray, psi1: np.ndarray, L, b) -> np.ndarray:
    """T0 psi1 (Eq. pro_mg) for one coarse field (V1, 2 Nv) -> fine field."""
    if psi1.ndim == 3:
        return np.stack([prolong(phi, p, L, b) for p in psi1])
    L = tuple(int(v) for v in L)
    sites = _lat.block_sites(L, b)
    V1, _, nv = phi.shape[:3]
    c1 = psi1.reshape(V1, 2, nv)
    loc = np.einsum("yac,yacksi->yksi", c1, phi)
    out = np.zeros((_lat.volume(L), 4, 3), dtype=np.complex128)
    out[sites] = loc
    return out.reshape(L + (4, 3))


def _crossing_mask(L, b, d: int) -> np.ndarray:
    """True at the sites whose hop in slot d leaves their block."""
    x = _lat.coords(L)
    mu = d % 4
    r = x[:, mu] % int(b[mu])
    if d < 4:
        m = r == int(b[mu]) - 1
    else:
        m = r == 0
    return m.reshape(tuple(int(v) for v in L))


def coarse_operator(U, phi, kappa, csw, b, bc_t=-1.0) -> np.ndarray:
    """Dhat[d, y, i, j], d = 0..8, as described in the module docstring:
    column j = (beta, c') is the restriction of D applied to T e_j split by
    hop slot."""
    L = tuple(int(v) for v in U.shape[:4])
    V1, _, nv = phi.shape[:3]
    n = 2 * nv
    A = _d.clover_matrix(U, kappa, csw)
    masks = [_crossing_mask(L, b, d)[..., None, None] for d in range(8)]
    Dhat = np.zeros((9, V1, n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((V1, n), dtype=np.complex128)
        e[:, j] = 1.0
        Phi = prolong(phi, e, L, b)  # phi_j on every block
        inside = _d.apply_clover(A, Phi)
        for d in range(8):
            h = _d.hop(U, Phi, d, bc_t)
            Dhat[d, :, :, j] = restrict(phi, np.where(masks[d], h, 0), L, b)
            inside += np.where(masks[d], 0, h)
        Dhat[8, :, :, j] = restrict(phi, inside, L, b)
    return Dhat


def coarse_apply(Dhat: np.ndarray, X: np.ndarray, Lb) -> np.ndarray:
    """Y(y) = sum_{d=0}^{8} Dhat[d, y] X(nbr_d(y)) for (V1, n) or a batch."""
    if X.ndim == 3:
        return np.stack([coarse_apply(Dhat, x, Lb) for x in X])
    nbr = _lat.coarse_neighbour_table(Lb)
    Y = np.zeros_like(X)
    for d in range(9):
        Y += np.einsum("yij,yj->yi", Dhat[d], X[nbr[:, d]])
    return Y


def coarse_apply_dagger(Dhat: np.ndarray, X: np.ndarray, Lb) -> np.ndarray:
    """The adjoint of ``coarse_apply``: Y(y') = sum_{d, y : nbr_d(y) = y'}
    Dhat[d, y]^dag X(y)."""
    if X.ndim == 3:
        return np.stack([coarse_apply_dagger(Dhat, x, Lb) for x in X])
    nbr = _lat.coarse_neighbour_table(Lb)
    Y = np.zeros_like(X)
    for d in range(9):
        contrib = np.einsum("yji,yj->yi", np.conj(Dhat[d]), X)
        np.add.at(Y, nbr[:, d], contrib)
    return Y


def coarse_gamma5(nv: int) -> np.ndarray:
    """gamma5 on a coarse site: +1 on alpha = 0 dofs, -1 on alpha = 1."""
    return np.concatenate([np.ones(nv), -np.ones(nv)])


def dense_coarse(Dhat: np.ndarray, Lb) -> np.ndarray:
    """The dense (V1 n x V1 n) matrix of the stencil (slots that land on the
    same block pair are summed)."""
    nbr = _lat.coarse_neighbour_table(Lb)
    V1, n = Dhat.shape[1], Dhat.shape[2]
    M = np.zeros((V1 * n, V1 * n), dtype=np.complex128)
    for d in range(9):
        for y in range(V1):
            z = nbr[y, d]
            M[y * n:(y + 1) * n, z * n:(z + 1) * n] += Dhat[d, y]
    return M


def dense_prolongator(phi: np.ndarray, L, b) -> np.ndarray:
    """The (12V x V1 n) matrix of T0, column j = T e_j."""
    L = tuple(int(v) for v in L)
    V1, _, nv = phi.shape[:3]
    n = 2 * nv
    cols = []
    for j in range(V1 * n):
        e = np.zeros(V1 * n, dtype=np.complex128)
        e[j] = 1
        cols.append(prolong(phi, e.reshape(V1, n), L, b).reshape(-1))
    return np.stack(cols, axis=1)


# ------------------------------------------------------------------ inner levels
def restrict_level(X: np.ndarray, Lb, b) -> np.ndarray:
    """R_l X for a coarse field X (V_l, n) on the grid Lb, blocks of side b
    (in level-l sites): sqrt(V_{l+1}/V_l) times the sum over each block."""
    if X.ndim == 3:
        return np.stack([restrict_level(x, Lb, b) for x in X])
    sites = _lat.block_sites(Lb, b)  # (V_{l+1}, |B|)
    f = np.sqrt(sites.shape[0] / _lat.volume(Lb))
    return f * X[sites].sum(axis=1)


def prolong_level(Y: np.ndarray, Lb, b) -> np.ndarray:
    """T_l Y for a field Y (V_{l+1}, n) of the next level: sqrt(V_{l+1}/V_l)
    times Y at the block of every level-l site."""
    if Y.ndim == 3:
        return np.stack([prolong_level(y, Lb, b) for y in Y])
    blk = _lat.block_of_site(Lb, b)
    f = np.sqrt(_lat.volume(_lat.block_grid(Lb, b)) / _lat.volume(Lb))
    return f * Y[blk]


def coarse_operator_next(Dhat: np.ndarray, Lb, b) -> np.ndarray:
    """D_{l+1} = R_l D_l T_l as the nine-slot stencil on the next grid, from
    the slot-wise stencil Dhat (9, V_l, n, n) of D_l (module docstring)."""
    Lb = tuple(int(v) for v in Lb)
    Lb2 = _lat.block_grid(Lb, b)
    V1, V2 = _lat.volume(Lb), _lat.volume(Lb2)
    n = Dhat.shape[2]
    blk = _lat.block_of_site(Lb, b)
    out = np.zeros((9, V2, n, n), dtype=np.complex128)
    f = V2 / V1
    leaves = [_crossing_mask(Lb, b, d).reshape(-1) for d in range(8)]
    for z in range(V1):
        y = blk[z]
        out[8, y] += f * Dhat[8, z]
        for d in range(8):
            # a hop that crosses the face of the next-level block keeps its
            # slot (the neighbour block may be y itself when the next grid has
            # extent 1 or 2 in that direction); one that stays inside is self
            out[d if leaves[d][z] else 8, y] += f * Dhat[d, z]
    return out


def dense_restrict_level(Lb, b) -> np.ndarray:
    """The (V_{l+1} n x V_l n) matrix of R_l for n = 1 (kron with 1_n for n
    dofs), row y, column z: sqrt(V_{l+1}/V_l) when z lies in B_y."""
    Lb2 = _lat.block_grid(Lb, b)
    V1, V2 = _lat.volume(Lb), _lat.volume(Lb2)
    R = np.zeros((V2, V1))
    R[_lat.block_of_site(Lb, b), np.arange(V1)] = np.sqrt(V2 / V1)
    return R


def multilevel_pieces(Dhats, Lbs, blocks, phi, L, b0, eta, tol=1e-13):
    """psi_l = T_l-compound D_l^-1 R_l-compound eta for l = 1 .. N-1 (Sec.
    "Multigrid decompositions", with Q_l^-1 R gamma5 replaced by D_l^-1 R by
    App. chirality): Dhats[l-1], Lbs[l-1] are the stencil and grid of level
    l, blocks[l-1] the blocking from level l to l+1 (len N-2), phi and b0 the
    level-1 basis and fine blocking.  The telescoping pieces are
    S_0 eta = x - psi_1, S_l eta = psi_l - psi_{l+1}, S_{N-1} eta = psi_{N-1}."""
    from . import solvers as _s
    r = restrict(phi, eta, L, b0)
    chain = [r]
    for l in range(1, len(Dhats)):
        chain.append(restrict_level(chain[-1], Lbs[l - 1], blocks[l - 1]))
    out = []
    for l in range(len(Dhats)):
        X, _, _ = _s.solve_coarse(Dhats[l], chain[l], Lbs[l], tol=tol)
        for k in range(l, 0, -1):
            X = prolong_level(X, Lbs[k - 1], blocks[k - 1])
        out.append(prolong(phi, X, L, b0))
    return out
