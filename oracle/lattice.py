"""Lattice geometry (oracle; test infrastructure only).

Sec. 3, Eqs. block_decomp / block_def / block_grid: the lattice
Lambda = {x | 0 <= x_mu < L_mu} is cut into disjoint blocks B_y of side b_mu,
y in Lambda_1 = {y | 0 <= y_mu < L_mu / b_mu}, with b_mu dividing L_mu.  The
block definition as printed gives only the upper bound x_mu - y_mu b_mu < b_mu;
the reading used here is 0 <= x_mu - y_mu b_mu < b_mu, i.e. y_mu = x_mu // b_mu.

Conventions (shared with the library): x0 is time; flat site index
((x0*L1 + x1)*L2 + x2)*L3 + x3; the block index and the site-in-block index
follow the same lexicographic rule on L/b and on x mod b; hop slot d = 0..3 is
+mu, 4..7 is -mu and 8 is the site itself.
"""
from __future__ import annotations

import itertools

import numpy as np


def volume(L) -> int:
    return int(np.prod([int(v) for v in L]))


def coords(L) -> np.ndarray:
    """Coordinates of every site, shape (V, 4), in flat-index order."""
    L = [int(v) for v in L]
    grid = np.indices(L).reshape(4, -1).T
    return grid.astype(np.int64)


def flat_index(x, L) -> np.ndarray:
    x = np.asarray(x, dtype=np.int64)
    return ((x[..., 0] * L[1] + x[..., 1]) * L[2] + x[..., 2]) * L[3] + x[..., 3]


def neighbour_table(L) -> np.ndarray:
    """nbr[i, d]: flat index of the neighbour of site i in hop slot d
    (d < 4: x + mu, 4 <= d < 8: x - mu, periodic), shape (V, 8), int32."""
    L = [int(v) for v in L]
    x = coords(L)
    out = np.empty((x.shape[0], 8), dtype=np.int32)
    for mu in range(4):
        for d, step in ((mu, +1), (mu + 4, -1)):
            y = x.copy()
            y[:, mu] = (y[:, mu] + step) % L[mu]
            out[:, d] = flat_index(y, L)
    return out


def check_blocking(L, b) -> None:
    for mu in range(4):
        if int(b[mu]) <= 0 or int(L[mu]) % int(b[mu]) != 0:
            raise ValueError(f"block side b[{mu}]={b[mu]} must divide L[{mu}]={L[mu]}")


def block_grid(L, b):
    check_blocking(L, b)
    return tuple(int(L[mu]) // int(b[mu]) for mu in range(4))


def block_of_site(L, b) -> np.ndarray:
    """Block index y(x) of every site (lexicographic on Lambda_1), int32."""
    Lb = block_grid(L, b)
    x = coords(L)
    y = x // np.asarray(b, dtype=np.int64)
    return flat_index(y, Lb).astype(np.int32)


def site_in_block(L, b) -> np.ndarray:
    """Index of every site inside its block (lexicographic on x mod b), int32."""
    x = coords(L)
    r = x % np.asarray(b, dtype=np.int64)
    return flat_index(r, [int(v) for v in b]).astype(np.int32)


def block_sites(L, b) -> np.ndarray:
    """sites[y, k]: flat index of the k-th site (site-in-block order) of block
    y, shape (V1, |B|), found by brute force over all coordinates."""
    Lb = block_grid(L, b)
    V1 = volume(Lb)
    nb = volume(b)
    out = np.empty((V1, nb), dtype=np.int64)
    bo = block_of_site(L, b)
    sib = site_in_block(L, b)
    out[bo, sib] = np.arange(volume(L))
    return out


def coarse_neighbour_table(Lb) -> np.ndarray:
    """Neighbours on the block grid, same slot convention, shape (V1, 9); slot
    8 is the block itself."""
    nb = neighbour_table(Lb)
    V1 = nb.shape[0]
    return np.concatenate([nb, np.arange(V1, dtype=np.int32)[:, None]], axis=1)


def brute_force_neighbours(L) -> np.ndarray:
    """The neighbour table by explicit loops over all coordinates (used to pin
    ``neighbour_table``)."""
    L = [int(v) for v in L]
    V = volume(L)
    out = np.empty((V, 8), dtype=np.int32)
    for x in itertools.product(*[range(n) for n in L]):
        i = ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]
        for mu in range(4):
            for d, s in ((mu, 1), (mu + 4, -1)):
                y = list(x)
                y[mu] = (y[mu] + s) % L[mu]
                out[i, d] = ((y[0] * L[1] + y[1]) * L[2] + y[2]) * L[3] + y[3]
    return out
