"""The shared input generators against published test vectors and their own
definitions; the paper's printed dimension ratios against the block geometry."""
import os

import numpy as np
import pytest

import synthetic
from oracle import lattice as lat

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors():
    # SplitMix64 reference outputs: seed 0 -> 0xE220A8397B1DCDAF; seed 1234567
    # gives 6457827717110365317, 3203168211198807973, ... (state += golden
    # ratio before each output).
    assert int(synthetic.mix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    g = 0x9E3779B97F4A7C15
    seq = [int(synthetic.mix64(np.uint64((1234567 + k * g) % 2**64))) for k in range(3)]
    assert seq == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_streams_are_counter_based():
    a = synthetic.stream_u64(5, 2, 0, 100)
    b = synthetic.stream_u64(5, 2, 40, 10)
    assert np.array_equal(a[40:50], b)
    u = synthetic.stream_uniform(5, 2, 0, 200000)
    assert u.min() > 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
    gs = synthetic.stream_gaussian(5, 3, 0, 200000)
    assert abs(gs.mean()) < 0.01 and abs(gs.var() - 1) < 0.02
    z = synthetic.z2_noise((2, 2, 2, 2), 3, 1)
    assert set(np.unique(z.real)) == {-1.0, 1.0} and np.all(z.imag == 0)
    z4 = synthetic.z4_noise((2, 2, 2, 2), 1, 1)
    assert np.allclose(np.abs(z4), 1.0)
    # first_rhs offsets select later RHS of the same stream
    assert np.array_equal(synthetic.z2_noise((2, 2, 2, 2), 3, 1)[2], synthetic.z2_noise((2, 2, 2, 2), 1, 1, first_rhs=2)[0])


def test_links_are_su3_and_match_expm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    L = (2, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.3, 7)
    uu = np.einsum("...ij,...kj->...ik", U, U.conj())
    assert np.allclose(uu, np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(U), 1, atol=1e-14)
    # link (site 3, mu 2) against scipy's expm of i eps H
    h = synthetic.stream_gaussian(7, synthetic.TAG_GAUGE, (3 * 4 + 2) * 8, 8)
    H = np.einsum("a,aij->ij", h, synthetic.gell_mann() / 2)
    assert np.allclose(H, H.conj().T) and abs(np.trace(H)) < 1e-15
    ref = scipy_linalg.expm(1j * 0.3 * H)
    assert np.allclose(U.reshape(-1, 4, 3, 3)[3, 2], ref, atol=1e-14)


def _golden_rows():
    rows, costs = [], []
    with open(os.path.join(GOLDEN, "paper_cost_model.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if "x" in parts[0]:
                rows.append(parts)
            else:
                costs.append(parts)
    return rows, costs


def test_paper_dimension_ratios_and_modelled_costs():
    rows, costs = _golden_rows()
    ratios = {}
    for r in rows:
        L = [int(v) for v in r[0].split("x")]
        b = [int(v) for v in r[1].split("x")]
        ns, nc, printed = int(r[2]), int(r[3]), float(r[4])
        fine = 12 * lat.volume(L)
        coarse = ns * nc * lat.volume(lat.block_grid(L, b))
        assert abs(fine / coarse - printed) < 1e-9
        ratios[tuple(b)] = fine / coarse
    # the printed modelled costs follow from cost = 4 sum_k N(Lk) / ratio(Lk)
    r8, r4 = ratios[(8, 8, 8, 8)], ratios[(4, 4, 4, 4)]
    for name, src, printed in costs:
        n = [int(v) for v in src.split(",")]
        per = [1.0] + ([r8] if len(n) == 2 else [r4, r8])
        cost = 4 * sum(ni / pi for ni, pi in zip(n, per))
        assert abs(cost - float(printed)) < 0.006, name
