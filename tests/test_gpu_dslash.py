"""GPU parity of the Wilson-clover stencil and its integer tables against the
FP64 oracle (through the C ABI).  Bars: integer tables bit-exact; FP64
operator applications within 1e-12 relative per RHS; FP32 within 2e-6."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from tests.gpu_util import rel_per_rhs, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2412_06347_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def ctx(m):
    c = m.Context(0)
    yield c
    c.close()


def load(m, ctx, L, eps, seed, kappa, csw, t_bc=-1):
    U = synthetic.gauge_links(L, eps, seed)
    return U, m.mglma_gauge_load(ctx, L, U, kappa, csw, t_bc=t_bc)


def oracle_op(U, psi, kappa, csw, op, t_bc=-1.0):
    out = []
    A = D.clover_matrix(U, kappa, csw)
    for p in psi:
        if op == 0:
            out.append(D.dirac(U, p, kappa, csw, t_bc, A))
        elif op == 1:
            out.append(D.dirac_dagger(U, p, kappa, csw, t_bc, A))
        elif op == 2:
            out.append(D.hermitian_dirac(U, p, kappa, csw, t_bc, A))
        else:
            out.append(D.dirac_dagger(U, D.dirac(U, p, kappa, csw, t_bc, A), kappa, csw, t_bc, A))
    return np.stack(out)


def test_tables_bit_exact(m, ctx):
    L, b = (6, 4, 2, 8), (2, 2, 1, 4)
    U, g = load(m, ctx, L, 0.3, 1, 0.12, 1.0)
    V = lat.volume(L)
    nbr = np.zeros((V, 8), dtype=np.int32)
    blk = np.zeros(V, dtype=np.int32)
    m.mglma_debug_tables(g, b, nbr, blk)
    assert np.array_equal(nbr, lat.neighbour_table(L))
    assert np.array_equal(blk, lat.block_of_site(L, b))
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("L,nrhs", [((8, 8, 8, 8), 3), ((6, 3, 5, 2), 5)])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_dirac_fp64_parity(m, ctx, L, nrhs, op):
    kappa, csw = 0.12, 1.0
    U, g = load(m, ctx, L, 0.3, 1001, kappa, csw)
    psi = np.concatenate([synthetic.z2_noise(L, 1, 3001), synthetic.random_spinors(L, nrhs - 1, 5)])
    out = np.zeros_like(psi)
    m.mglma_dirac_apply(ctx, g, op, nrhs, psi, out, m.MGLMA_FP64)
    ref = oracle_op(U, psi, kappa, csw, op)
    assert rel_per_rhs(out, ref).max() < 1e-12
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("L,nrhs", [((8, 8, 8, 8), 4), ((6, 3, 5, 2), 7)])
def test_dirac_fp32_parity(m, ctx, L, nrhs):
    kappa, csw = 0.125, 1.7
    U, g = load(m, ctx, L, 0.2, 1002, kappa, csw)
    psi = synthetic.random_spinors(L, nrhs, 6)
    for op in (0, 1, 2):
        out = np.zeros_like(psi)
        m.mglma_dirac_apply(ctx, g, op, nrhs, psi, out, m.MGLMA_FP32)
        assert rel_per_rhs(out, oracle_op(U, psi, kappa, csw, op)).max() < 2e-6
    m.mglma_gauge_free(g)


TILES = [(1, 1), (2, 1), (4, 1), (1, 2), (1, 4), (2, 2), (2, 4), ("staged", 4), ("staged", 8), ("staged", 16)]


def tile_code(m, nr, rw):
    return m.dslash32_staged_code(rw) if nr == "staged" else m.dslash32_tile_code(nr, rw)


@pytest.mark.parametrize("nr,rw", TILES)
def test_dirac_fp32_tile_shapes(m, ctx, nr, rw):
    """Every FP32 tile shape (RHS per thread x RHS tiles per CTA, and the
    staged-tile kernel's 32 sites x NRT RHS) against the oracle, with RHS
    counts that leave partial tiles and partial tile groups and a volume
    (6x3x5x2 = 180) that is not a multiple of any CTA's sites."""
    kappa, csw = 0.125, 1.7
    L = (6, 3, 5, 2)
    U, g = load(m, ctx, L, 0.2, 1002, kappa, csw)
    c = m.Context(0)
    for nrhs in (1, 5, 11, 17):
        m.mglma_autotune_set(c, 0, nrhs, tile_code(m, nr, rw))
        psi = synthetic.random_spinors(L, nrhs, 60 + nrhs)
        for op in (0, 1, 2, 3):
            out = np.zeros_like(psi)
            m.mglma_dirac_apply(c, g, op, nrhs, psi, out, m.MGLMA_FP32)
            assert rel_per_rhs(out, oracle_op(U, psi, kappa, csw, op)).max() < 2e-6, (nrhs, op)
    c.close()
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("L,t_bc", [((6, 3, 5, 2), -1), ((4, 4, 4, 8), 1), ((2, 8, 2, 16), -1)])
def test_staged_kernel_equals_thread_per_site_bitwise(m, ctx, L, t_bc):
    """The staged-tile kernel pre-scales the staged links by -1/2 (times
    t_bc across the time boundary), which is exact, and sums the terms in the
    order of the one-site-per-thread kernel: both give identical bits for D,
    D^dag, Q and D^dag D."""
    kappa, csw = 0.1266, 1.9
    U = synthetic.gauge_links(L, 0.2, 1005)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw, t_bc=t_bc)
    c = m.Context(0)
    nrhs = 9
    psi = synthetic.random_spinors(L, nrhs, 70)
    for op in (0, 1, 2, 3):
        outs = []
        for code in (m.dslash32_tile_code(1, 1), m.dslash32_staged_code(4), m.dslash32_staged_code(8),
                     m.dslash32_staged_code(16)):
            m.mglma_autotune_set(c, 0, nrhs, code)
            o = np.zeros_like(psi)
            m.mglma_dirac_apply(c, g, op, nrhs, psi, o, m.MGLMA_FP32)
            outs.append(o)
        for o in outs[1:]:
            assert np.array_equal(o, outs[0]), op
    c.close()
    m.mglma_gauge_free(g)


def test_autotune_set_rejects_unknown(m, ctx):
    with pytest.raises(m.MglmaError):
        m.mglma_autotune_set(ctx, 0, 4, m.dslash32_tile_code(4, 2))
    with pytest.raises(m.MglmaError):
        m.mglma_autotune_set(ctx, 1, 4, 12)


@pytest.mark.parametrize("L,eps,seed,t_bc", [((8, 8, 8, 8), 0.3, 1001, -1), ((6, 4, 2, 10), 0.15, 1004, 1)])
def test_device_gauge_generator_matches_host(m, ctx, L, eps, seed, t_bc):
    """mglma_gauge_random draws the links of synthetic.gauge_links on the
    device; D built from them equals D from the host links to rounding."""
    kappa, csw = 0.1266, 1.9
    U = synthetic.gauge_links(L, eps, seed)
    g_host = m.mglma_gauge_load(ctx, L, U, kappa, csw, t_bc=t_bc)
    g_dev = m.mglma_gauge_random(ctx, L, eps, seed, kappa, csw, t_bc=t_bc)
    psi = synthetic.random_spinors(L, 2, 9)
    a, b = np.zeros_like(psi), np.zeros_like(psi)
    m.mglma_dirac_apply(ctx, g_host, 0, 2, psi, a, m.MGLMA_FP64)
    m.mglma_dirac_apply(ctx, g_dev, 0, 2, psi, b, m.MGLMA_FP64)
    assert rel_per_rhs(b, a).max() < 1e-13
    assert rel_per_rhs(a, oracle_op(U, psi, kappa, csw, 0, t_bc=float(t_bc))).max() < 1e-12
    m.mglma_gauge_free(g_host)
    m.mglma_gauge_free(g_dev)


def test_periodic_time_bc_and_free_field(m, ctx):
    L = (4, 4, 4, 4)
    U = synthetic.free_links(L)
    g = m.mglma_gauge_load(ctx, L, U, 0.13, 1.9, t_bc=+1)
    psi = synthetic.random_spinors(L, 2, 8)
    out = np.zeros_like(psi)
    m.mglma_dirac_apply(ctx, g, 0, 2, psi, out, m.MGLMA_FP64)
    assert rel_per_rhs(out, oracle_op(U, psi, 0.13, 1.9, 0, t_bc=+1.0)).max() < 1e-13
    m.mglma_gauge_free(g)


def test_device_pointers_stream_and_slabs(m, ctx):
    import torch
    L = (8, 4, 4, 6)
    U = synthetic.gauge_links(L, 0.3, 77)
    g1 = m.mglma_gauge_load(ctx, L, U, 0.12, 1.3)
    # slab loading: two slabs in reverse order give identical bits
    Uf = U.reshape(L[0], -1)
    g2 = m.mglma_gauge_load(ctx, L, np.ascontiguousarray(Uf[5:]), 0.12, 1.3, t_begin=5, t_count=3)
    g2 = m.mglma_gauge_load(ctx, L, np.ascontiguousarray(Uf[:5]), 0.12, 1.3, t_begin=0, t_count=5, gauge=g2)
    psi = synthetic.random_spinors(L, 3, 9)
    host = np.zeros_like(psi)
    m.mglma_dirac_apply(ctx, g1, 0, 3, psi, host, m.MGLMA_FP64)
    dpsi = to_device(psi)
    dout = torch.zeros_like(dpsi)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())  # the copies and the zero fill come first
    with torch.cuda.stream(s):
        m.mglma_dirac_apply(ctx, g2, 0, 3, dpsi, dout, m.MGLMA_FP64, stream=s)
    s.synchronize()
    assert np.array_equal(dout.cpu().numpy(), host)
    m.mglma_gauge_free(g1)
    m.mglma_gauge_free(g2)


def test_non_su3_links_rejected(m, ctx):
    L = (2, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.3, 5)
    U[1, 0, 1, 1, 2] *= 1.001
    with pytest.raises(m.MglmaError) as e:
        m.mglma_gauge_load(ctx, L, U, 0.12, 1.0)
    assert e.value.status == 1


def test_full_size_sampled_sites(m, ctx):
    """64x32^3 (the 2 fm box shape), eps 0.15, kappa 0.1266, csw 1.9: the
    FP64 and FP32 stencils on a Z2 source against the oracle evaluated site by
    site at sampled sites, plus gamma5-hermiticity over the whole lattice."""
    L, kappa, csw = (64, 32, 32, 32), 0.1266, 1.9
    U, g = load(m, ctx, L, 0.15, 1004, kappa, csw)
    eta = synthetic.z2_noise(L, 1, 3004)
    V = lat.volume(L)
    sites = np.concatenate([[0, V - 1, 31, 32 * 32 * 32 * 63], synthetic.point_source_sites(L, 12, 99)])
    ref = D.dirac_at_sites(U, eta[0], kappa, csw, sites)
    for prec, tol in ((m.MGLMA_FP64, 1e-12), (m.MGLMA_FP32, 2e-6)):
        out = np.zeros_like(eta)
        m.mglma_dirac_apply(ctx, g, 0, 1, eta, out, prec)
        got = out[0].reshape(V, 4, 3)[sites]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    chi = synthetic.random_spinors(L, 1, 12)
    a, b = np.zeros_like(chi), np.zeros_like(eta)
    m.mglma_dirac_apply(ctx, g, 2, 1, eta, b, m.MGLMA_FP64)
    m.mglma_dirac_apply(ctx, g, 2, 1, chi, a, m.MGLMA_FP64)
    lhs, rhs = np.vdot(chi, b), np.vdot(a, eta)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    m.mglma_gauge_free(g)


def test_sources_bit_exact(m, ctx):
    """Device sources equal the host generator bit for bit (same counter
    definition); point sources and time dilution."""
    L = (6, 4, 2, 4)
    z2 = np.zeros((3,) + L + (4, 3), dtype=np.complex128)
    m.mglma_sources(ctx, L, m.MGLMA_SOURCE_Z2, 3, 77, z2, first=2)
    assert np.array_equal(z2, synthetic.z2_noise(L, 3, 77, first_rhs=2))
    z4 = np.zeros_like(z2)
    m.mglma_sources(ctx, L, m.MGLMA_SOURCE_Z4, 3, 78, z4)
    assert np.array_equal(z4, synthetic.z4_noise(L, 3, 78))
    td = np.zeros_like(z2)
    m.mglma_sources(ctx, L, m.MGLMA_SOURCE_Z4, 3, 78, td, t_slice=4)
    ref = synthetic.z4_noise(L, 3, 78)
    ref[:, :4] = 0
    ref[:, 5:] = 0
    assert np.array_equal(td, ref)
    pt = np.zeros_like(z2)
    sites = [0, 17, lat.volume(L) - 1]
    m.mglma_sources(ctx, L, m.MGLMA_SOURCE_POINT, 3, 0, pt, point_sites=sites, point_sc=[0, 5, 11])
    ref = np.concatenate([synthetic.point_sources(L, [s], sc) for s, sc in zip(sites, [0, 5, 11])])
    assert np.array_equal(pt, ref)
