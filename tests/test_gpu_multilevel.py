"""GPU parity of the deeper levels of the hierarchy (Sec. "Multigrid
decompositions") against the FP64 oracle: the aggregated operator
D_{l+1} = R_l D_l T_l, the inner-level transfers R_l / T_l, the level-l
stencil applied in FP64 and in BF16 on tensor cores, and the pieces
calT_l D_l^-1 calR_l b of the telescoping decomposition, on 8^4 with 2^4
blocks (level 1 on 4^4), then 2^4 blocks of level-1 sites (level 2 on 2^4),
then one block of everything (level 3: one site, the LMA limit)."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG
from tests.gpu_util import rel_per_rhs

pytestmark = pytest.mark.gpu

L, B0, NV, KAPPA, CSW = (8, 8, 8, 8), (2, 2, 2, 2), 8, 0.12, 1.0
BLOCKS = [(2, 2, 2, 2), (2, 2, 2, 2)]


@pytest.fixture(scope="module")
def m():
    import paper_2412_06347_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def hier(m):
    ctx = m.Context(0)
    U = synthetic.gauge_links(L, 0.3, 1001)
    g = m.mglma_gauge_load(ctx, L, U, KAPPA, CSW)
    sub = m.mglma_subspace_build(ctx, g, B0, NV, 5, 2001, m.MGLMA_FP64)
    C = [m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)]
    for b in BLOCKS:
        C.append(m.mglma_coarse_build_next(ctx, C[-1], b, m.MGLMA_BF16))
    Lbs = [lat.block_grid(L, B0)]
    for b in BLOCKS:
        Lbs.append(lat.block_grid(Lbs[-1], b))
    # the oracle's own chain from the same seeded starts
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, NV, 2001), KAPPA, CSW, B0, 5)
    Dh = [MG.coarse_operator(U, phi, KAPPA, CSW, B0)]
    for l, b in enumerate(BLOCKS):
        Dh.append(MG.coarse_operator_next(Dh[-1], Lbs[l], b))
    yield dict(ctx=ctx, U=U, g=g, sub=sub, C=C, Lbs=Lbs, phi=phi, Dh=Dh)
    for c in reversed(C):
        m.mglma_coarse_free(c)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)
    ctx.close()


def export(m, c, Lb):
    out = np.zeros((9, lat.volume(Lb), 2 * NV, 2 * NV), dtype=np.complex128)
    m.mglma_coarse_export(c, out)
    return out


def test_aggregated_operator_matches_oracle(m, hier):
    for l in (1, 2):
        nv, Lb, V = m.mglma_coarse_info(hier["C"][l])
        assert nv == NV and Lb == tuple(hier["Lbs"][l]) and V == lat.volume(Lb)
        parent = export(m, hier["C"][l - 1], hier["Lbs"][l - 1])
        got = export(m, hier["C"][l], hier["Lbs"][l])
        # the aggregation of the GPU's own parent stencil (FP64 sums: exact to rounding)
        ref = MG.coarse_operator_next(parent, hier["Lbs"][l - 1], BLOCKS[l - 1])
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        # and the oracle's whole chain from its own basis (the basis agrees to 1e-11)
        assert np.abs(got - hier["Dh"][l]).max() <= 1e-10 * np.abs(hier["Dh"][l]).max()
    assert hier["Lbs"][2] == (1, 1, 1, 1)


def test_level_transfers(m, hier):
    ctx = hier["ctx"]
    for l in (1, 2):
        Lb, b = hier["Lbs"][l - 1], BLOCKS[l - 1]
        V, V2 = lat.volume(Lb), lat.volume(hier["Lbs"][l])
        X = synthetic.random_coarse(V, 2 * NV, 3, 31 + l)
        out = np.zeros((3, V2, 2 * NV), dtype=np.complex128)
        m.mglma_coarse_restrict(ctx, hier["C"][l], 3, X, out)
        assert rel_per_rhs(out, MG.restrict_level(X, Lb, b)).max() < 1e-14
        Y = synthetic.random_coarse(V2, 2 * NV, 2, 41 + l)
        back = np.zeros((2, V, 2 * NV), dtype=np.complex128)
        m.mglma_coarse_prolong(ctx, hier["C"][l], 2, Y, back)
        assert rel_per_rhs(back, MG.prolong_level(Y, Lb, b)).max() < 1e-14
    with pytest.raises(m.MglmaError):  # level 1 has no inner-level transfer
        m.mglma_coarse_restrict(ctx, hier["C"][0], 1, np.zeros((1, 256, 16), np.complex128),
                                np.zeros((1, 16, 16), np.complex128))


@pytest.mark.parametrize("op", [0, 1, 2])
def test_level_apply_fp64_and_tensor_cores(m, hier, op):
    ctx = hier["ctx"]
    for l in (1, 2):
        Lb = hier["Lbs"][l]
        Dh = export(m, hier["C"][l], Lb)
        X = synthetic.random_coarse(lat.volume(Lb), 2 * NV, 5, 51 + l)
        g5 = MG.coarse_gamma5(NV)
        xin = X * g5 if op == 1 else X
        ref = MG.coarse_apply(Dh, xin, Lb)
        if op in (1, 2):
            ref = ref * g5
        for prec, tol in ((m.MGLMA_FP64, 1e-13), (m.MGLMA_FP32, 2e-2)):
            out = np.zeros_like(X)
            m.mglma_coarse_apply(ctx, hier["C"][l], 5, X, out, prec, op=op)
            assert rel_per_rhs(out, ref).max() < tol, (l, prec)


def test_multilevel_pieces(m, hier):
    ctx = hier["ctx"]
    b = synthetic.z2_noise(L, 2, 3001)
    psi = np.zeros((3,) + b.shape, dtype=np.complex128)
    m.mglma_pieces(ctx, hier["g"], hier["C"], 2, b, psi, tol=1e-12)
    for i in range(2):
        ref = MG.multilevel_pieces(hier["Dh"], hier["Lbs"], BLOCKS, hier["phi"], L, B0, b[i], tol=1e-13)
        for l in range(3):
            err = np.linalg.norm(psi[l, i] - ref[l]) / np.linalg.norm(ref[l])
            assert err < 1e-8, (i, l, err)
    # with x = D^-1 b the outer pieces S_0 + ... + S_{l-1} = x - psi_l are
    # Galerkin-orthogonal on level l: calR_l D (x - psi_l) = 0
    x = np.zeros_like(b)
    xc = np.zeros_like(b)
    m.mglma_solve_batch(ctx, hier["g"], hier["C"][0], m.mglma_solve_params_default(m.MGLMA_SOLVER_MG), [2], b, x,
                        xc)
    for i in range(2):
        r = D.dirac(hier["U"], x[i] - psi[0, i], KAPPA, CSW)
        c = MG.restrict(hier["phi"], r, L, B0)
        ref = np.linalg.norm(MG.restrict(hier["phi"], b[i], L, B0))
        for l in range(3):
            assert np.linalg.norm(c) < 1e-8 * ref, (i, l)
            if l < 2:
                r = D.dirac(hier["U"], x[i] - psi[l + 1, i], KAPPA, CSW)
                c = MG.restrict(hier["phi"], r, L, B0)
                for k in range(l + 1):
                    c = MG.restrict_level(c, hier["Lbs"][k], BLOCKS[k])
    # psi_1 of the hierarchy equals the two-level piece of mglma_solve_batch
    assert rel_per_rhs(psi[0], xc).max() < 1e-8
