"""Solves at the benchmark configurations' full sizes, judged by the FP64
oracle's own residual ||b - D x|| / ||b|| of the GPU's x (evaluated in time
slabs, ``oracle.solvers.residual_slabs``, or site by site where only a sample
is affordable):

* 32x16^3 (eps 0.2, kappa 0.125, csw 1.7, 4^4 blocks, Nv 16): one Z2 source,
  the plain FP64 CGNE (complex128 throughout) against the mixed multigrid
  solve (complex64 inner FGCR, BF16 coarse stencil, FP64 defect correction);
  both reach 1e-10 in the oracle's residual and agree with each other.
* 48x24^3 (eps 0.2, kappa 0.1265, csw 1.9, 4^4 blocks, Nv 20): three seeded
  ragged groups with sizes in 1..64, merged into lockstep batches; every RHS
  converged with the library's FP64 residual, sampled RHS checked by the
  oracle, and RHS solved alone equal their batched results.
* 64x32^3 (eps 0.15, kappa 0.1266, csw 1.9, 4^4 blocks, Nv 24 with 5 MR + 60
  FP32 CG relaxation, FP16 basis, BF16 coarse stencil): a point and a Z2
  source of the benchmark's set, oracle residual <= 1e-10.
"""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import solvers as S

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


def test_c2_fp64_cgne_vs_mixed(m, ctx):
    L, kappa, csw = (32, 16, 16, 16), 0.125, 1.7
    U = synthetic.gauge_links(L, 0.2, 1002)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_create(ctx, g, (4, 4, 4, 4), 16, 5, 2002, m.MGLMA_FP32, n_cg=60, cg_prec=m.MGLMA_FP32)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    b = synthetic.z2_noise(L, 1, 3002)
    x64 = np.zeros_like(b)
    xmg = np.zeros_like(b)
    _, s64 = m.mglma_solve_batch(ctx, g, None, m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE), [1], b, x64)
    _, smg = m.mglma_solve_batch(ctx, g, C, m.mglma_solve_params_default(m.MGLMA_SOLVER_MG), [1], b, xmg)
    A = D.clover_matrix(U, kappa, csw)
    r64 = S.true_residual(U, x64[0], b[0], kappa, csw, A=A)
    rmg = S.true_residual(U, xmg[0], b[0], kappa, csw, A=A)
    assert r64 <= 1e-10 and rmg <= 1e-10, (r64, rmg)
    # the library's own FP64 residual agrees with the oracle's
    assert abs(smg[0]["residual"] - rmg) <= 1e-3 * rmg + 1e-14
    # the two solutions of the unique x = D^-1 b agree (both residuals 1e-10,
    # times the condition number of D)
    assert np.linalg.norm(x64 - xmg) / np.linalg.norm(x64) < 1e-6
    # the mixed solve needs far fewer fine operator applications
    assert smg[0]["iterations"] < s64[0]["iterations"] / 4
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_c3_ragged_groups_1_to_64(m, ctx):
    import torch
    L, kappa, csw = (48, 24, 24, 24), 0.1265, 1.9
    U = synthetic.gauge_links(L, 0.2, 1003)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_create(ctx, g, (4, 4, 4, 4), 20, 5, 2003, m.MGLMA_FP32, n_cg=60, cg_prec=m.MGLMA_FP32)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    groups = [int(v) for v in synthetic.ragged_groups(3, 1, 64, 4013)]
    n = sum(groups)
    V = lat.volume(L)
    # Z2 sources generated on the device (bit-exact with synthetic.z2_noise)
    b = torch.empty((n, V, 12), dtype=torch.complex128, device="cuda")
    m.mglma_sources(ctx, L, m.MGLMA_SOURCE_Z2, n, 3003, b)
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG)
    _, st = m.mglma_solve_batch(ctx, g, C, prm, groups, b, x)
    assert all(s["converged"] and s["residual"] <= 1e-10 for s in st)
    assert max(s["batch"] for s in st) > 1  # RHS of different groups shared launches
    # oracle residuals: the first RHS of every group in full, every RHS at
    # sampled sites
    firsts = np.cumsum([0] + groups[:-1])
    bf = np.stack([synthetic.z2_noise(L, 1, 3003, first_rhs=int(i))[0] for i in firsts])
    xf = np.stack([x[int(i)].cpu().numpy().reshape(L + (4, 3)) for i in firsts])
    assert S.residual_slabs(U, xf, bf, kappa, csw, slab=6).max() <= 1e-10
    sites = synthetic.point_source_sites(L, 4, 6)
    xs = x.reshape(n, V, 4, 3)
    for i in range(n):
        loc = xs[i].cpu().numpy().reshape(L + (4, 3))
        bi = b[i].reshape(V, 4, 3)[torch.as_tensor(sites, device="cuda")].cpu().numpy()
        r = D.dirac_at_sites(U, loc, kappa, csw, sites) - bi
        assert np.abs(r).max() <= 1e-10 * np.sqrt(12 * V)
    # batch-equals-alone: the last RHS of the first group and the first of the last
    for i in (int(firsts[1]) - 1, int(firsts[-1])):
        xi = torch.zeros_like(x[i:i + 1])
        m.mglma_solve_batch(ctx, g, C, prm, [1], b[i:i + 1], xi)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(xi[0] - x[i]) / torch.linalg.norm(x[i])).item() <= 1e-9
    del b, x
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_c4_bench_solve_oracle_residual(m, ctx):
    L, kappa, csw = (64, 32, 32, 32), 0.1266, 1.9
    U = synthetic.gauge_links(L, 0.15, 1004)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_create(ctx, g, (4, 4, 4, 4), 24, 5, 2004, m.MGLMA_FP16, n_cg=60, cg_prec=m.MGLMA_FP32)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    site = synthetic.point_source_sites(L, 4, 3004)[:1]
    b = np.concatenate([synthetic.point_sources(L, site, 5), synthetic.z2_noise(L, 1, 3004)])
    x = np.zeros_like(b)
    _, st = m.mglma_solve_batch(ctx, g, C, m.mglma_solve_params_default(m.MGLMA_SOLVER_MG), [2], b, x)
    assert all(s["converged"] for s in st)
    res = S.residual_slabs(U, x, b, kappa, csw, slab=4)
    for i in range(2):
        assert res[i] <= 1e-10, (i, res[i])
        assert abs(st[i]["residual"] - res[i]) <= 1e-3 * res[i] + 1e-14
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)
