"""GPU parity of the block basis, R0/T0, the coarse operator and its
application against the FP64 oracle.  The oracle builds its own basis from the
same seeded start vectors (the counter-based generator both sides implement);
the factor is unique, so the two agree to rounding.  Bars: FP64 to 1e-11
(basis, Gram-Schmidt conditioning) / 1e-12 (operators); FP32 to 2e-6; FP16
basis to 2e-3; BF16 operator to 2e-2."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
from oracle import lattice as lat
from oracle import multigrid as MG
from tests.gpu_util import rel_per_rhs

pytestmark = pytest.mark.gpu

CASES = {
    # name: L, block, nv, eps, seed, kappa, csw, n_smooth
    "c1": ((8, 8, 8, 8), (2, 2, 2, 2), 8, 0.3, 1001, 0.12, 1.0, 5),
    "ragged": ((6, 4, 6, 2), (3, 2, 2, 1), 5, 0.3, 7, 0.125, 1.7, 3),
    "lma": ((4, 2, 2, 4), (4, 2, 2, 4), 4, 0.3, 9, 0.125, 1.9, 2),
}


@pytest.fixture(scope="module")
def m():
    import paper_2412_06347_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def ctx(m):
    c = m.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module", params=list(CASES))
def setup(request, m, ctx):
    L, b, nv, eps, seed, kappa, csw, ns = CASES[request.param]
    U = synthetic.gauge_links(L, eps, seed)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_build(ctx, g, b, nv, ns, seed + 1000, m.MGLMA_FP64)
    starts = synthetic.gaussian_start_vectors(L, nv, seed + 1000)
    phi = MG.subspace(U, starts, kappa, csw, b, ns)
    yield dict(L=L, b=b, nv=nv, U=U, g=g, sub=sub, phi=phi, kappa=kappa, csw=csw, seed=seed)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_basis_matches_oracle(m, setup):
    s = setup
    phi = np.zeros_like(s["phi"])
    m.mglma_subspace_export(s["sub"], phi)
    assert np.linalg.norm(phi - s["phi"]) / np.linalg.norm(s["phi"]) < 1e-11
    nv, Lb, V1 = m.mglma_subspace_info(s["sub"])
    assert nv == s["nv"] and V1 == lat.volume(lat.block_grid(s["L"], s["b"]))


def test_restrict_prolong_fp64(m, ctx, setup):
    s = setup
    L, b, phi = s["L"], s["b"], s["phi"]
    psi = synthetic.random_spinors(L, 3, 21)
    V1 = phi.shape[0]
    out = np.zeros((3, V1, 2 * s["nv"]), dtype=np.complex128)
    m.mglma_restrict(ctx, s["sub"], 3, psi, out, m.MGLMA_FP64)
    assert rel_per_rhs(out, MG.restrict(phi, psi, L, b)).max() < 1e-11
    c = synthetic.random_coarse(V1, 2 * s["nv"], 2, 22)
    f = np.zeros((2,) + tuple(L) + (4, 3), dtype=np.complex128)
    m.mglma_prolong(ctx, s["sub"], 2, c, f, m.MGLMA_FP64)
    assert rel_per_rhs(f, MG.prolong(phi, c, L, b)).max() < 1e-11


def test_coarse_operator_and_apply(m, ctx, setup):
    s = setup
    L, b = s["L"], s["b"]
    Lb = lat.block_grid(L, b)
    V1, n2 = lat.volume(Lb), 2 * s["nv"]
    Dhat_ref = MG.coarse_operator(s["U"], s["phi"], s["kappa"], s["csw"], b)
    for store, tol in ((m.MGLMA_FP64, 2e-6), (m.MGLMA_FP32, 2e-6), (m.MGLMA_BF16, 2e-2)):
        C = m.mglma_coarse_build(ctx, s["g"], s["sub"], store)
        Dh = np.zeros((9, V1, n2, n2), dtype=np.complex128)
        m.mglma_coarse_export(C, Dh)
        assert np.linalg.norm(Dh - Dhat_ref) / np.linalg.norm(Dhat_ref) < 1e-11
        X = synthetic.random_coarse(V1, n2, 9, 23)
        ref = MG.coarse_apply(Dhat_ref, X, Lb)
        Y = np.zeros_like(X)
        m.mglma_coarse_apply(ctx, C, 9, X, Y, m.MGLMA_FP64)
        assert rel_per_rhs(Y, ref).max() < 1e-12
        m.mglma_coarse_apply(ctx, C, 9, X, Y, m.MGLMA_FP32)
        assert rel_per_rhs(Y, ref).max() < tol
        # Q1 = g5hat D1 and D1^dag = g5hat D1 g5hat against the oracle's
        # stencil transpose (gamma5-hermiticity of the coarse operator)
        g5 = MG.coarse_gamma5(s["nv"])
        dag = MG.coarse_apply_dagger(Dhat_ref, X, Lb)
        for op, want in ((m.MGLMA_OP_Q, g5 * ref), (m.MGLMA_OP_DDAG, dag)):
            m.mglma_coarse_apply(ctx, C, 9, X, Y, m.MGLMA_FP64, op=op)
            assert rel_per_rhs(Y, want).max() < 1e-11
            m.mglma_coarse_apply(ctx, C, 9, X, Y, m.MGLMA_FP32, op=op)
            assert rel_per_rhs(Y, want).max() < tol
        with pytest.raises(m.MglmaError):
            m.mglma_coarse_apply(ctx, C, 9, X, Y, m.MGLMA_FP64, op=m.MGLMA_OP_DDAGD)
        m.mglma_coarse_free(C)


@pytest.mark.parametrize("nv,nrhs", [(6, 5), (8, 17)])
def test_low_precision_transfers(m, ctx, nv, nrhs):
    """FP32 R0 / T0 against the oracle on the same basis; (8, 17) runs the
    many-RHS kernels (tiles of 16 RHS, a one-RHS remainder tile), (6, 5) the
    few-RHS ones."""
    L, b = (8, 4, 4, 8), (4, 4, 4, 4)
    U = synthetic.gauge_links(L, 0.2, 31)
    g = m.mglma_gauge_load(ctx, L, U, 0.125, 1.7)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 32), 0.125, 1.7, b, 2)
    psi = synthetic.random_spinors(L, nrhs, 33)
    ref = MG.restrict(phi, psi, L, b)
    c = synthetic.random_coarse(phi.shape[0], 2 * nv, nrhs, 34)
    pref = MG.prolong(phi, c, L, b)
    for store, tol in ((m.MGLMA_FP32, 2e-6), (m.MGLMA_FP16, 2e-3)):
        sub = m.mglma_subspace_build(ctx, g, b, nv, 2, 32, store)
        out = np.zeros_like(ref)
        m.mglma_restrict(ctx, sub, nrhs, psi, out, m.MGLMA_FP32)
        assert rel_per_rhs(out, ref).max() < tol
        f = np.zeros_like(psi)
        m.mglma_prolong(ctx, sub, nrhs, c, f, m.MGLMA_FP32)
        assert rel_per_rhs(f, pref).max() < tol
        m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("nv,nrhs", [(8, 16), (8, 17), (24, 16)])
def test_tensor_core_restrict(m, ctx, nv, nrhs):
    """R0 on the tensor cores (BF16 operands, FP32 accumulation) against the
    oracle on the same basis: 4^4 blocks (four 64-site segments per component
    pair), one or two RHS tiles, FP32 and FP16 stored bases.  The bound is the
    BF16 rounding of both operands (2^-9 each) summed over the block."""
    L, b = (8, 4, 4, 8), (4, 4, 4, 4)
    U = synthetic.gauge_links(L, 0.2, 31)
    g = m.mglma_gauge_load(ctx, L, U, 0.125, 1.7)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 32), 0.125, 1.7, b, 2)
    psi = synthetic.random_spinors(L, nrhs, 35)
    ref = MG.restrict(phi, psi, L, b)
    for store in (m.MGLMA_FP32, m.MGLMA_FP16):
        sub = m.mglma_subspace_build(ctx, g, b, nv, 2, 32, store)
        out = np.zeros_like(ref)
        m.mglma_restrict(ctx, sub, nrhs, psi, out, m.MGLMA_BF16)
        err = rel_per_rhs(out, ref)
        assert err.max() < 1e-2 and err.min() > 0, (store, err.max())
        m.mglma_subspace_free(sub)
    # Nv = 6 is not a multiple of 8: refused before any device work
    sub = m.mglma_subspace_build(ctx, g, b, 6, 2, 32, m.MGLMA_FP32)
    with pytest.raises(m.MglmaError) as e:
        m.mglma_restrict(ctx, sub, 2, psi[:2], np.zeros((2, ref.shape[1], 12), ref.dtype), m.MGLMA_BF16)
    assert e.value.status == 1
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("nv,nrhs,b", [(8, 16, (4, 4, 4, 4)), (8, 17, (4, 4, 4, 4)), (24, 16, (4, 4, 4, 4)),
                                       (16, 33, (2, 4, 4, 4))])
def test_tensor_core_prolong(m, ctx, nv, nrhs, b):
    """T0 on the tensor cores (BF16 coarse fields and basis image, FP32
    accumulation) against the oracle on the same basis: 256-site blocks (two
    128-row tiles per component) and 128-site blocks, full and ragged RHS
    tiles, FP32 and FP16 stored bases.  The bound is the BF16 rounding of both
    operands summed over the 2 Nv coarse dofs."""
    L = (8, 4, 4, 8)
    U = synthetic.gauge_links(L, 0.2, 31)
    g = m.mglma_gauge_load(ctx, L, U, 0.125, 1.7)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 32), 0.125, 1.7, b, 2)
    c = synthetic.random_coarse(phi.shape[0], 2 * nv, nrhs, 36)
    ref = MG.prolong(phi, c, L, b)
    for store in (m.MGLMA_FP32, m.MGLMA_FP16):
        sub = m.mglma_subspace_build(ctx, g, b, nv, 2, 32, store)
        f = np.full(ref.shape, 7.0 + 0j, ref.dtype)  # overwritten, not accumulated
        m.mglma_prolong(ctx, sub, nrhs, c, f, m.MGLMA_BF16)
        err = rel_per_rhs(f, ref)
        assert err.max() < 1e-2 and err.min() > 0, (store, err.max())
        m.mglma_subspace_free(sub)
    # 64-site blocks fill no 128-row tile, Nv = 6 no K chunk: both refused
    # before any device work
    for bb, n in (((4, 4, 2, 2), 8), (b, 6)):
        sub = m.mglma_subspace_build(ctx, g, bb, n, 2, 32, m.MGLMA_FP32)
        nc = lat.volume(L) // int(np.prod(bb))
        with pytest.raises(m.MglmaError) as e:
            m.mglma_prolong(ctx, sub, 2, np.zeros((2, nc, 2 * n), complex), np.zeros((2,) + ref.shape[1:], ref.dtype),
                            m.MGLMA_BF16)
        assert e.value.status == 1
        m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_subspace_load_exact_modes_and_rank_error(m, ctx):
    """Basis from caller-given vectors (exact low modes of Q, Sec. 3) and the
    rank check on linearly dependent vectors."""
    L, b, nv = (4, 2, 2, 2), (2, 2, 2, 2), 3
    U = synthetic.gauge_links(L, 0.4, 61)
    kappa, csw = 0.125, 1.5
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    M = D.dense_dirac(U, kappa, csw)
    G5 = np.kron(np.eye(lat.volume(L)), np.kron(D.gamma5(), np.eye(3)))
    w, v = np.linalg.eigh(G5 @ M)
    order = np.argsort(np.abs(w))[:nv]
    modes = np.ascontiguousarray(v[:, order].T.reshape((nv,) + L + (4, 3)))
    sub = m.mglma_subspace_load(ctx, g, b, nv, modes, m.MGLMA_FP64)
    phi = np.zeros_like(MG.build_basis(modes, L, b))
    m.mglma_subspace_export(sub, phi)
    assert np.linalg.norm(phi - MG.build_basis(modes, L, b)) < 1e-11 * np.linalg.norm(phi)
    m.mglma_subspace_free(sub)
    bad = np.ascontiguousarray(np.stack([modes[0], modes[1], modes[0] * (2 - 1j)]))
    with pytest.raises(m.MglmaError) as e:
        m.mglma_subspace_load(ctx, g, b, nv, bad, m.MGLMA_FP64)
    assert e.value.status == 4
    m.mglma_gauge_free(g)


def test_basis_with_cg_relaxation(m, ctx):
    """Set-up with MR then CG relaxation on D x = 0 (FP64) against the
    oracle's recipe from the same seeded starts."""
    L, b, nv, kappa, csw = (8, 4, 4, 8), (2, 2, 2, 4), 4, 0.125, 1.7
    U = synthetic.gauge_links(L, 0.2, 41)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_create(ctx, g, b, nv, 3, 42, m.MGLMA_FP64, n_cg=12, cg_prec=m.MGLMA_FP64)
    ref = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 42), kappa, csw, b, 3, n_cg=12)
    phi = np.zeros_like(ref)
    m.mglma_subspace_export(sub, phi)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-10
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("nrhs", [1, 5, 8, 16, 21, 40])
def test_coarse_tensor_core_apply(m, ctx, nrhs):
    """BF16 operator on tcgen05 (FP32 accumulation) for ragged RHS tiles,
    against the oracle's FP64 stencil application: relative error at the
    BF16 operand level (<= 2e-2 per RHS)."""
    L, b, nv, kappa, csw = (8, 8, 4, 8), (2, 2, 2, 2), 8, 0.125, 1.7
    U = synthetic.gauge_links(L, 0.2, 51)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_build(ctx, g, b, nv, 2, 52, m.MGLMA_FP64)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    phi = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 52), kappa, csw, b, 2)
    Lb = lat.block_grid(L, b)
    Dh = MG.coarse_operator(U, phi, kappa, csw, b)
    X = synthetic.random_coarse(lat.volume(Lb), 2 * nv, nrhs, 53)
    Y = np.zeros_like(X)
    m.mglma_coarse_apply(ctx, C, nrhs, X, Y, m.MGLMA_FP32)
    err = rel_per_rhs(Y, MG.coarse_apply(Dh, X, Lb))
    assert err.max() < 2e-2 and err.min() > 0
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


def test_coarse_tensor_core_full_size_properties(m, ctx):
    """64x32^3 with 4^4 blocks and Nv 24 (8192 coarse sites, 48 dofs): the
    tensor-core application agrees with the FP64 application of the same
    operator to BF16 accuracy, and <X, g5 D1 Y> = <g5 D1 X, Y> holds."""
    L, b, nv = (64, 32, 32, 32), (4, 4, 4, 4), 24
    U = synthetic.gauge_links(L, 0.15, 1004)
    g = m.mglma_gauge_load(ctx, L, U, 0.1266, 1.9)
    del U
    sub = m.mglma_subspace_build(ctx, g, b, nv, 2, 2004, m.MGLMA_FP16)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    nv_, Lb, V1 = m.mglma_coarse_info(C)
    X = synthetic.random_coarse(V1, 2 * nv, 3, 61)
    Y32, Y64 = np.zeros_like(X), np.zeros_like(X)
    m.mglma_coarse_apply(ctx, C, 3, X, Y32, m.MGLMA_FP32)
    m.mglma_coarse_apply(ctx, C, 3, X, Y64, m.MGLMA_FP64)
    assert rel_per_rhs(Y32, Y64).max() < 2e-2
    g5 = MG.coarse_gamma5(nv)
    lhs = np.vdot(X[0], g5 * Y64[1])
    rhs = np.vdot(g5 * Y64[0], X[1])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs32 = np.vdot(X[0], g5 * Y32[1])
    rhs32 = np.vdot(g5 * Y32[0], X[1])
    assert abs(lhs32 - rhs32) <= 2e-2 * abs(lhs32)
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)


@pytest.mark.parametrize("store,btol", [("fp32", 1e-4), ("fp16", 3e-3)])
def test_lean_subspace_coarse_and_solve(m, ctx, store, btol):
    """Memory-lean set-up (FP32 test vectors relaxed three at a time, FP64
    orthonormalisation on chunks of blocks, no FP64 basis copy): the stored
    basis is the oracle's recipe to the storage precision and orthonormal per
    (block, chirality); FP64 R0 / T0 and the coarse operator built from it
    equal the oracle's definitions applied to the same stored basis; after
    the FP64 operator is released the MG solve still reaches 1e-10."""
    from oracle import solvers as S
    prec = {"fp32": m.MGLMA_FP32, "fp16": m.MGLMA_FP16}[store]
    L, b, nv, kappa, csw = (8, 8, 8, 8), (2, 2, 2, 2), 8, 0.125, 1.7
    U = synthetic.gauge_links(L, 0.2, 71)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_create(ctx, g, b, nv, 3, 72, prec, n_cg=4, lean_group=3)
    ref = MG.subspace(U, synthetic.gaussian_start_vectors(L, nv, 72), kappa, csw, b, 3, n_cg=4)
    phi = np.zeros_like(ref)
    m.mglma_subspace_export(sub, phi)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < btol
    V1, nB = phi.shape[0], phi.shape[3]
    for y in (0, V1 // 2, V1 - 1):
        for a in range(2):
            Q = phi[y, a].reshape(nv, -1)
            assert np.abs(Q.conj() @ Q.T - np.eye(nv)).max() < 4 * btol
    # FP64 transfers on the stored basis
    psi = synthetic.random_spinors(L, 2, 73)
    out = np.zeros((2, V1, 2 * nv), dtype=np.complex128)
    m.mglma_restrict(ctx, sub, 2, psi, out, m.MGLMA_FP64)
    assert rel_per_rhs(out, MG.restrict(phi, psi, L, b)).max() < 1e-12
    f = np.zeros_like(psi)
    m.mglma_prolong(ctx, sub, 2, out, f, m.MGLMA_FP64)
    assert rel_per_rhs(f, MG.prolong(phi, out, L, b)).max() < 1e-12
    # coarse operator of the stored basis
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    Dh = np.zeros((9, V1, 2 * nv, 2 * nv), dtype=np.complex128)
    m.mglma_coarse_export(C, Dh)
    Dref = MG.coarse_operator(U, phi, kappa, csw, b)
    assert np.linalg.norm(Dh - Dref) / np.linalg.norm(Dref) < 1e-12
    m.mglma_coarse_release_fp64(C)
    with pytest.raises(m.MglmaError):
        m.mglma_coarse_export(C, Dh)
    bsrc = synthetic.z2_noise(L, 3, 74)
    x = np.zeros_like(bsrc)
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG)
    _, st = m.mglma_solve_batch(ctx, g, C, prm, [3], bsrc, x)
    assert all(s["converged"] for s in st)
    A = D.clover_matrix(U, kappa, csw)
    assert max(S.true_residual(U, xi, bi, kappa, csw, A=A) for xi, bi in zip(x, bsrc)) <= 1e-10
    with pytest.raises(m.MglmaError):  # the pieces need the FP64 basis
        m.mglma_solve_batch(ctx, g, C, prm, [3], bsrc, x, x_coarse=np.zeros((3, V1, 2 * nv), np.complex128))
    m.mglma_coarse_free(C)
    m.mglma_subspace_free(sub)
    m.mglma_gauge_free(g)
