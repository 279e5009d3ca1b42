"""GPU parity of the even-odd (Schur) preconditioned coarse operator against
the FP64 oracle: S_ee = D_ee - D_eo D_oo^-1 D_oe and g5hat S_ee through the
C ABI in FP64 (composed FP64 applications) and FP32 (three parity-restricted
launches of the tensor-core stencil, BF16 operands), the multigrid solve with
MINRES on g5hat S_ee as the preconditioner's coarse solver reaching the
oracle's 1e-10 residual, and the refusal of a coarse grid with an odd
extent."""
import numpy as np
import pytest

import synthetic
from oracle import lattice as lat
from oracle import multigrid as MG
from oracle import solvers as S
from tests.gpu_util import rel_per_rhs

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


@pytest.fixture(scope="module")
def c1(m, ctx):
    L, b, nv, kappa, csw = (8, 8, 8, 8), (2, 2, 2, 2), 8, 0.12, 1.0
    U = synthetic.gauge_links(L, 0.3, 1001)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_build(ctx, g, b, nv, 5, 2001, m.MGLMA_FP64)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    Lb = lat.block_grid(L, b)
    Dh = np.zeros((9, lat.volume(Lb), 2 * nv, 2 * nv), dtype=np.complex128)
    m.mglma_coarse_export(C, Dh)
    yield dict(L=L, b=b, nv=nv, kappa=kappa, csw=csw, U=U, g=g, sub=sub, C=C, Lb=Lb, Dh=Dh)
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("op", ["schur", "schur_q"])
def test_schur_apply_matches_oracle(m, ctx, c1, op):
    Lb, nv = c1["Lb"], c1["nv"]
    V1, n2 = lat.volume(Lb), 2 * nv
    par = S.parity(Lb)
    Se = S.schur_even(MG.dense_coarse(c1["Dh"], Lb), par, n2)
    if op == "schur_q":
        Se = np.tile(MG.coarse_gamma5(nv), V1 // 2)[:, None] * Se
    X = synthetic.random_coarse(V1, n2, 3, 61)
    e = par == 0
    ref = np.stack([(Se @ x[e].reshape(-1)).reshape(-1, n2) for x in X])
    code = m.MGLMA_OP_SCHUR if op == "schur" else m.MGLMA_OP_SCHUR_Q
    for prec, tol in ((m.MGLMA_FP64, 1e-12), (m.MGLMA_FP32, 2e-2)):
        out = np.full_like(X, np.nan)
        m.mglma_coarse_apply(ctx, c1["C"], 3, X, out, prec, op=code)
        assert np.all(out[:, ~e] == 0)
        assert rel_per_rhs(out[:, e], ref).max() < tol, prec


def test_mg_solve_with_even_odd_coarse_minres(m, ctx, c1):
    b = synthetic.z2_noise(c1["L"], 3, 3021)
    res = {}
    for name, cs in (("minres", m.MGLMA_COARSE_MINRES), ("minres_eo", m.MGLMA_COARSE_MINRES_EO)):
        x = np.zeros_like(b)
        prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG, coarse_solver=cs)
        _, st = m.mglma_solve_batch(ctx, c1["g"], c1["C"], prm, [3], b, x)
        assert all(s["converged"] for s in st)
        r = S.residual_slabs(c1["U"], x, b, c1["kappa"], c1["csw"], slab=8)
        assert r.max() <= 1e-10
        res[name] = (x, max(s["iterations"] for s in st))
    # the same unique solution
    assert rel_per_rhs(res["minres"][0], res["minres_eo"][0]).max() < 1e-8
    # the Schur system is no worse a preconditioner than the full one
    assert res["minres_eo"][1] <= 1.5 * res["minres"][1]


def test_odd_coarse_extent_rejected(m, ctx):
    L = (6, 4, 6, 2)
    U = synthetic.gauge_links(L, 0.3, 7)
    g = m.mglma_gauge_load(ctx, L, U, 0.125, 1.7)
    sub = m.mglma_subspace_build(ctx, g, (3, 2, 2, 1), 4, 3, 8, m.MGLMA_FP64)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_FP64)
    X = np.zeros((1, lat.volume(lat.block_grid(L, (3, 2, 2, 1))), 8), dtype=np.complex128)
    with pytest.raises(m.MglmaError) as e:
        m.mglma_coarse_apply(ctx, C, 1, X, np.zeros_like(X), m.MGLMA_FP64, op=m.MGLMA_OP_SCHUR)
    assert e.value.status == 1 and "even" in str(e.value)
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("op", ["schur", "schur_q"])
def test_fine_schur_matches_oracle(m, ctx, op):
    """The fine even-odd operator S = A_ee - H_eo A_oo^-1 H_oe (FP64, clover
    inverses formed on the device) against the dense oracle on 4x2x2x2."""
    from oracle import dirac as D
    L, kappa, csw = (4, 2, 2, 2), 0.124, 1.3
    U = synthetic.gauge_links(L, 0.3, 95)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    par = S.parity(L)
    Se = S.schur_even(D.dense_dirac(U, kappa, csw), par, 12)
    e = par == 0
    if op == "schur_q":
        g5 = np.kron(np.eye(lat.volume(L)), np.kron(D.gamma5(), np.eye(3)))
        Se = g5[np.ix_(np.repeat(e, 12), np.repeat(e, 12))] @ Se
    psi = synthetic.random_spinors(L, 2, 96)
    out = np.full_like(psi, np.nan)
    m.mglma_dirac_apply(ctx, g, m.MGLMA_OP_SCHUR if op == "schur" else m.MGLMA_OP_SCHUR_Q, 2, psi, out, m.MGLMA_FP64)
    flat_in = psi.reshape(2, -1, 12)
    flat_out = out.reshape(2, -1, 12)
    ref = np.stack([(Se @ v[e].reshape(-1)).reshape(-1, 12) for v in flat_in])
    assert np.all(flat_out[:, ~e] == 0)
    assert rel_per_rhs(flat_out[:, e], ref).max() < 1e-13
    m.mglma_gauge_free(g)


def test_fine_schur_gamma5_hermitian_8x8x8x8(m, ctx, c1):
    """<chi, gamma5 S psi> = <gamma5 S chi, psi> on the even sites of 8^4."""
    a = synthetic.random_spinors(c1["L"], 2, 97)
    Sa = np.zeros_like(a)
    m.mglma_dirac_apply(ctx, c1["g"], m.MGLMA_OP_SCHUR_Q, 2, a, Sa, m.MGLMA_FP64)
    e = (S.parity(c1["L"]) == 0).reshape(c1["L"])
    lhs = np.vdot(a[0][e], Sa[1][e])
    rhs = np.vdot(Sa[0][e], a[1][e])
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_cgne_even_odd_solve(m, ctx, c1):
    b = synthetic.z2_noise(c1["L"], 2, 3041)
    x_eo = np.zeros_like(b)
    x_cg = np.zeros_like(b)
    _, s_eo = m.mglma_solve_batch(ctx, c1["g"], None, m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE_EO), [2], b,
                                  x_eo)
    _, s_cg = m.mglma_solve_batch(ctx, c1["g"], None, m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE), [2], b, x_cg)
    assert all(s["converged"] for s in s_eo)
    r = S.residual_slabs(c1["U"], x_eo, b, c1["kappa"], c1["csw"], slab=8)
    assert r.max() <= 1e-10
    assert rel_per_rhs(x_eo, x_cg).max() < 1e-8
    # the Schur system needs fewer CG iterations than the full normal equations
    assert max(s["iterations"] for s in s_eo) < max(s["iterations"] for s in s_cg)
