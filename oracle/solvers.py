"""Krylov solves and propagator pieces (oracle; test infrastructure only).

* The propagator S = D^-1 is unique, so ``cgne`` -- the conjugate-gradient
  method (Hestenes-Stiefel) on the normal equations D^dag D x = D^dag b, the
  plain method -- is only a way to reach it; it stops when the recursively
  updated residual of D x = b satisfies ||r|| / ||b|| <= tol.
* Sec. 2: S = S0 + S1 with S1 = T Q1^-1 R gamma5, Q1 = R Q T, Q = gamma5 D;
  App. chirality: with [P, gamma5] = 0 this equals T D1^-1 R with
  D1 = R D T.  ``pieces`` returns psi = S eta, psi1 = T D1^-1 R eta and
  psi0 = psi - psi1.
"""
from __future__ import annotations

import numpy as np

from . import dirac as _d
from . import multigrid as _mg


def _vdot(a, b):
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def _norm2(a):
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


def cgne(apply, apply_dag, b, tol=1e-11, maxiter=100000, x0=None):
    """CG on D^dag D x = D^dag b.  Returns (x, iterations, final ||r||/||b||)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x) if x0 is not None else b.copy()
    bn = np.sqrt(_norm2(b))
    if bn == 0:
        return x, 0, 0.0
    z = apply_dag(r)
    p = z.copy()
    zz = _norm2(z)
    it = 0
    while np.sqrt(_norm2(r)) / bn > tol and it < maxiter:
        w = apply(p)
        a = zz / _norm2(w)
        x += a * p
        r -= a * w
        z = apply_dag(r)
        zz_new = _norm2(z)
        p = z + (zz_new / zz) * p
        zz = zz_new
        it += 1
    return x, it, np.sqrt(_norm2(r)) / bn


def solve_fine(U, b, kappa, csw, bc_t=-1.0, tol=1e-11, maxiter=100000, A=None):
    """x = D^-1 b for one field by ``cgne``."""
    if A is None:
        A = _d.clover_matrix(U, kappa, csw)
    f = lambda v: _d.dirac(U, v, kappa, csw, bc_t, A)  # noqa: E731
    g = lambda v: _d.dirac_dagger(U, v, kappa, csw, bc_t, A)  # noqa: E731
    return cgne(f, g, b, tol, maxiter)


def solve_coarse(Dhat, b1, Lb, tol=1e-12, maxiter=100000):
    """X = D1^-1 b1 for one coarse field by ``cgne``."""
    f = lambda v: _mg.coarse_apply(Dhat, v, Lb)  # noqa: E731
    g = lambda v: _mg.coarse_apply_dagger(Dhat, v, Lb)  # noqa: E731
    return cgne(f, g, b1, tol, maxiter)


def true_residual(U, x, b, kappa, csw, bc_t=-1.0, A=None) -> float:
    """||b - D x|| / ||b|| in FP64."""
    r = b - _d.dirac(U, x, kappa, csw, bc_t, A)
    return float(np.sqrt(_norm2(r) / _norm2(b)))


def _slab_slices(L0: int, t0: int, t1: int) -> np.ndarray:
    """Time slices t0 - 1 .. t1 (mod L0): the slab [t0, t1) with one halo
    slice on each side."""
    return np.arange(t0 - 1, t1 + 1) % L0


def dirac_slab(U, psi, kappa, csw, t0: int, t1: int, bc_t=-1.0, A=None) -> np.ndarray:
    """(D psi)(x) for the time slices t0 <= x0 < t1 of one field, from the
    links and spinors of slices t0 - 1 .. t1 only.  Every term of D at x
    (the clover leaves and the hops) touches slices x0 - 1 .. x0 + 1, so D is
    evaluated by ``dirac`` on the extended slab taken as periodic, and the two
    halo results -- the only ones that see the artificial wrap -- are dropped.
    The fermion boundary sign is carried by the halo spinors instead: a halo
    slice that lies across the lattice's time boundary (t0 = 0 below, t1 = L0
    above) enters multiplied by bc_t, and the slab is then applied with
    periodic hops.  A (optional) is the clover matrix of the extended slab's
    links, ``dirac.clover_matrix(U[slices t0 - 1 .. t1])``."""
    L0 = U.shape[0]
    idx = _slab_slices(L0, t0, t1)
    Us = U[idx]
    ps = psi[idx].copy()
    if t0 == 0:
        ps[0] *= bc_t
    if t1 == L0:
        ps[-1] *= bc_t
    out = _d.dirac(Us, ps, kappa, csw, 1.0, A)
    return out[1:-1]


def residual_slabs(U, x, b, kappa, csw, bc_t=-1.0, slab=4):
    """||b - D x|| / ||b|| in FP64, D evaluated ``slab`` time slices at a
    time (``dirac_slab``), so the clover term and the work arrays never cover
    more than slab + 2 slices: the oracle's check of a solution on lattices
    too large for ``true_residual``.  x, b: one field, or a batch (n, L...,
    4, 3) sharing each slab's clover term; returns a float, or n floats."""
    one = x.ndim == 6
    xs, bs = (x[None], b[None]) if one else (x, b)
    L0 = U.shape[0]
    rr = np.zeros(len(xs))
    for t0 in range(0, L0, slab):
        t1 = min(L0, t0 + slab)
        A = _d.clover_matrix(U[_slab_slices(L0, t0, t1)], kappa, csw)
        for i in range(len(xs)):
            rr[i] += _norm2(bs[i][t0:t1] - dirac_slab(U, xs[i], kappa, csw, t0, t1, bc_t, A))
    res = np.sqrt(rr / np.array([_norm2(v) for v in bs]))
    return float(res[0]) if one else res


def pieces(U, phi, Dhat, eta, kappa, csw, b, bc_t=-1.0, tol=1e-11):
    """(psi, psi1, psi0) for one source eta: psi = D^-1 eta,
    psi1 = T D1^-1 R eta, psi0 = psi - psi1."""
    L = U.shape[:4]
    Lb = tuple(int(L[m]) // int(b[m]) for m in range(4))
    psi, _, _ = solve_fine(U, eta, kappa, csw, bc_t, tol)
    X, _, _ = solve_coarse(Dhat, _mg.restrict(phi, eta, L, b), Lb, tol * 0.1)
    psi1 = _mg.prolong(phi, X, L, b)
    return psi, psi1, psi - psi1


# ------------------------------------------------------------------ even-odd (Schur) preconditioning
def parity(L) -> np.ndarray:
    """(x0 + x1 + x2 + x3) mod 2 of every site, flat site order."""
    from . import lattice as _lat
    return (_lat.coords(L).sum(axis=1) % 2).astype(np.int64)


def eo_blocks(M: np.ndarray, par: np.ndarray, ndof: int):
    """The four parity blocks (ee, eo, oe, oo) of a dense operator M on sites
    with `ndof` components each (site-major), sites ordered as in `par`."""
    e = np.repeat(par == 0, ndof)
    o = ~e
    return M[np.ix_(e, e)], M[np.ix_(e, o)], M[np.ix_(o, e)], M[np.ix_(o, o)]


def schur_even(M: np.ndarray, par: np.ndarray, ndof: int) -> np.ndarray:
    """S_ee = M_ee - M_eo M_oo^-1 M_oe, the Schur complement on the even sites
    (the even-odd preconditioned operator when every hop joins sites of
    opposite parity, which holds when every lattice extent is even; the paper
    applies it to the coarse operator, Sec. "Comparison of the cost")."""
    Mee, Meo, Moe, Moo = eo_blocks(M, par, ndof)
    return Mee - Meo @ np.linalg.solve(Moo, Moe)


def solve_eo(M: np.ndarray, par: np.ndarray, ndof: int, b: np.ndarray) -> np.ndarray:
    """x = M^-1 b through the Schur complement: S_ee x_e = b_e - M_eo M_oo^-1 b_o,
    then x_o = M_oo^-1 (b_o - M_oe x_e) (dense solves)."""
    Mee, Meo, Moe, Moo = eo_blocks(M, par, ndof)
    e = np.repeat(par == 0, ndof)
    be, bo = b[e], b[~e]
    xe = np.linalg.solve(Mee - Meo @ np.linalg.solve(Moo, Moe), be - Meo @ np.linalg.solve(Moo, bo))
    xo = np.linalg.solve(Moo, bo - Moe @ xe)
    x = np.empty_like(b)
    x[e], x[~e] = xe, xo
    return x
