"""Seeded synthetic inputs shared by the FP64 oracle and the tests of the CUDA path.

This module holds input generation only -- gauge links, noise and point
sources, random start vectors, random gauge transformations, batch-size and
arrival draws -- and none of the arithmetic of the multigrid method itself.

Every random number comes from one counter-based generator so that any slice
of a field can be regenerated independently and the CUDA library can draw the
same numbers on the device:

* SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014) is the mixing function ``mix64``.
* A stream is keyed by ``key = mix64(mix64(seed) ^ tag)``; its n-th 64-bit
  draw is ``mix64(key + n)`` (all arithmetic modulo 2^64).
* A uniform double in (0, 1) is ``((z >> 11) + 0.5) * 2^-53``.
* Gaussians come in Box--Muller pairs: draws 2k and 2k+1 give u1, u2 and
  ``r = sqrt(-2 ln u1)``; element 2k is ``r cos(2 pi u2)`` and element 2k+1 is
  ``r sin(2 pi u2)``.

Lattice conventions: coordinates x = (x0, x1, x2, x3) with x0 the time
direction; arrays are shaped (L0, L1, L2, L3, ...) in C order, so a flat site
index is ((x0*L1 + x1)*L2 + x2)*L3 + x3.  Spinors are (..., 4 spins, 3
colours) complex128; links are (..., 4 directions mu, 3, 3) with U_mu(x) on
the link x -> x + mu.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "TAG_GAUGE", "TAG_NOISE", "TAG_START", "TAG_POINT", "TAG_GAUGE_TRANSFORM",
    "TAG_GROUPS", "TAG_ARRIVALS", "TAG_FIELD",
    "mix64", "stream_u64", "stream_uniform", "stream_gaussian",
    "gell_mann", "gauge_links", "random_su3", "z2_noise", "z4_noise",
    "point_sources", "gaussian_start_vectors", "random_spinors",
    "ragged_groups", "poisson_arrivals", "free_links",
]

# Stream tags: one independent stream per kind of input.
TAG_GAUGE = 1
TAG_NOISE = 2
TAG_START = 3
TAG_POINT = 4
TAG_GAUGE_TRANSFORM = 5
TAG_GROUPS = 6
TAG_ARRIVALS = 7
TAG_FIELD = 8

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    """SplitMix64 output function applied to uint64 values (wrapping)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, tag: int) -> np.uint64:
    return mix64(mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF)) ^ np.uint64(tag))


def stream_u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of stream (seed, tag)."""
    k = _key(seed, tag)
    with np.errstate(over="ignore"):
        n = np.arange(start, start + count, dtype=np.uint64)
        return mix64(k + n)


def stream_uniform(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    z = stream_u64(seed, tag, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def stream_gaussian(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Gaussians start .. start+count-1; start and count must be even."""
    assert start % 2 == 0 and count % 2 == 0
    u = stream_uniform(seed, tag, start, count).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    phi = 2.0 * np.pi * u[:, 1]
    out = np.empty((u.shape[0], 2))
    out[:, 0] = r * np.cos(phi)
    out[:, 1] = r * np.sin(phi)
    return out.reshape(-1)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _expi_project(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps H) by an order-18 Taylor series (Horner form), then projected
    onto SU(3): rows 0 and 1 by Gram--Schmidt, row 2 = conj(row0 x row1).
    The batched 3x3 products run through torch's CPU matmul for speed."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(1j * eps * h))
    eye = torch.eye(3, dtype=torch.complex128)
    u = eye.expand_as(x).clone()
    for k in range(18, 0, -1):
        u = torch.matmul(x, u).div_(k).add_(eye)
    u = u.numpy()
    r0 = u[..., 0, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _su3_from_stream(seed: int, tag: int, first: int, count: int, eps: float) -> np.ndarray:
    """count SU(3) matrices exp(i eps H), H = sum_a h_a lambda_a / 2 with
    h_a ~ N(0, 1) taken from Gaussians (first + j)*8 + a of the stream."""
    h = stream_gaussian(seed, tag, first * 8, count * 8).reshape(count, 8)
    lam = (gell_mann() / 2.0).reshape(8, 9)
    hm = (h.astype(np.complex128) @ lam).reshape(count, 3, 3)
    return _expi_project(hm, eps)


def gauge_links(L, eps: float, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """Random SU(3) links U_mu(x) = P_SU3(exp(i eps H)), one Gaussian traceless
    Hermitian H per link; link (site, mu) uses stream index site*4 + mu.
    Returns complex128 (L0, L1, L2, L3, 4, 3, 3)."""
    L = tuple(int(v) for v in L)
    n = int(np.prod(L)) * 4
    out = np.empty((n, 3, 3), dtype=np.complex128)

    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        out[s:s + c] = _su3_from_stream(seed, TAG_GAUGE, s, c, eps)
    return out.reshape(L + (4, 3, 3))


def free_links(L) -> np.ndarray:
    """Unit links, complex128 (L0, L1, L2, L3, 4, 3, 3)."""
    L = tuple(int(v) for v in L)
    u = np.zeros(L + (4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def random_su3(L, eps: float, seed: int) -> np.ndarray:
    """One random SU(3) matrix per site (a gauge transformation), shape
    (L0, L1, L2, L3, 3, 3)."""
    L = tuple(int(v) for v in L)
    n = int(np.prod(L))
    return _su3_from_stream(seed, TAG_GAUGE_TRANSFORM, 0, n, eps).reshape(L + (3, 3))


def z2_noise(L, nrhs: int, seed: int, first_rhs: int = 0) -> np.ndarray:
    """Z2 noise: each real component is +1 or -1 (imaginary part 0), from bit
    63 of draw (rhs*V + site)*12 + spin*3 + colour.  Shape (nrhs, L..., 4, 3)."""
    L = tuple(int(v) for v in L)
    per = int(np.prod(L)) * 12
    z = stream_u64(seed, TAG_NOISE, first_rhs * per, nrhs * per)
    v = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
    return v.astype(np.complex128).reshape((nrhs,) + L + (4, 3))


def z4_noise(L, nrhs: int, seed: int, first_rhs: int = 0) -> np.ndarray:
    """Z4 noise {+-1 +- i}/sqrt(2): bits 63 and 62 of the same draws as
    ``z2_noise`` give the signs of the real and imaginary parts."""
    L = tuple(int(v) for v in L)
    per = int(np.prod(L)) * 12
    z = stream_u64(seed, TAG_NOISE, first_rhs * per, nrhs * per)
    re = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
    im = np.where(((z >> np.uint64(62)) & np.uint64(1)) == 0, 1.0, -1.0)
    return ((re + 1j * im) / np.sqrt(2.0)).reshape((nrhs,) + L + (4, 3))


def point_sources(L, sites, spin_colour=None) -> np.ndarray:
    """Point sources: for each (site, spin*3+colour) pair a unit vector.  With
    ``spin_colour`` None every site gives its 12 spin-colour columns."""
    L = tuple(int(v) for v in L)
    V = int(np.prod(L))
    cols = []
    for s in sites:
        for sc in (range(12) if spin_colour is None else [spin_colour]):
            cols.append((int(s), int(sc)))
    out = np.zeros((len(cols), V, 12), dtype=np.complex128)
    for r, (s, sc) in enumerate(cols):
        out[r, s, sc] = 1.0
    return out.reshape((len(cols),) + L + (4, 3))


def point_source_sites(L, count: int, seed: int) -> np.ndarray:
    """Sites for point sources, drawn uniformly from stream TAG_POINT."""
    V = int(np.prod([int(v) for v in L]))
    z = stream_u64(seed, TAG_POINT, 0, count)
    return (z % np.uint64(V)).astype(np.int64)


def gaussian_start_vectors(L, nv: int, seed: int) -> np.ndarray:
    """Random starts for the test vectors: complex component k = spin*3 +
    colour of vector c at site s has real/imaginary parts given by the
    Gaussian pair (2n, 2n+1) with n = (c*V + s)*12 + k of stream TAG_START.
    Shape (nv, L..., 4, 3).  The CUDA library draws the same numbers on the
    device from the same definition."""
    L = tuple(int(v) for v in L)
    per = int(np.prod(L)) * 12
    g = stream_gaussian(seed, TAG_START, 0, 2 * nv * per).reshape(-1, 2)
    return (g[:, 0] + 1j * g[:, 1]).reshape((nv,) + L + (4, 3))


def random_spinors(L, nrhs: int, seed: int, tag: int = TAG_FIELD) -> np.ndarray:
    """Generic Gaussian complex test fields, same recipe as the start vectors
    but on stream ``tag``."""
    L = tuple(int(v) for v in L)
    per = int(np.prod(L)) * 12
    g = stream_gaussian(seed, tag, 0, 2 * nrhs * per).reshape(-1, 2)
    return (g[:, 0] + 1j * g[:, 1]).reshape((nrhs,) + L + (4, 3))


def random_coarse(nsites: int, ndof: int, nrhs: int, seed: int, tag: int = TAG_FIELD) -> np.ndarray:
    """Gaussian complex coarse fields, shape (nrhs, nsites, ndof)."""
    n = nrhs * nsites * ndof
    g = stream_gaussian(seed, tag, 0, 2 * n).reshape(-1, 2)
    return (g[:, 0] + 1j * g[:, 1]).reshape(nrhs, nsites, ndof)


def ragged_groups(n_groups: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Group sizes uniform in [lo, hi] (inclusive), one per group."""
    z = stream_u64(seed, TAG_GROUPS, 0, n_groups)
    return (lo + (z % np.uint64(hi - lo + 1))).astype(np.int64)


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate:
    cumulative sums of exponential gaps -ln(u)/rate."""
    u = stream_uniform(seed, TAG_ARRIVALS, 0, n)
    return np.cumsum(-np.log(u) / rate)


def uniform_ints(n: int, lo: int, hi: int, seed: int, tag: int) -> np.ndarray:
    """n integers uniform in [lo, hi] from stream ``tag``."""
    z = stream_u64(seed, tag, 0, n)
    return (lo + (z % np.uint64(hi - lo + 1))).astype(np.int64)
