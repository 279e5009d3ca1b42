"""GPU parity of the time-slice contraction of the stochastic estimator
(Sec. 5, Eq. C_stoch2) and of its gamma5 gamma_k sources against the oracle,
and the whole estimator (sources -> FP64 solves -> contraction) against the
trace formula of Eq. tmr on a dense inverse."""
import numpy as np
import pytest

import synthetic
from oracle import contract as K
from oracle import dirac as D
from tests.gpu_util import to_device

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


@pytest.mark.parametrize("L,nrhs", [((6, 3, 5, 2), 3), ((8, 8, 8, 8), 2), ((4, 16, 16, 8), 1)])
def test_contract_parity(m, ctx, L, nrhs):
    a = synthetic.random_spinors(L, 3 * nrhs, 81).reshape((nrhs, 3) + tuple(L) + (4, 3))
    b = synthetic.random_spinors(L, nrhs, 82)
    out = np.zeros((nrhs, L[0]), dtype=np.complex128)
    m.mglma_contract(ctx, L, nrhs, a, b, out)
    for r in range(nrhs):
        ref = K.slice_correlator(a[r], b[r])
        assert np.abs(out[r] - ref).max() <= 1e-12 * np.abs(ref).max()
    # device buffers give the same bits (written in order on the context's
    # stream: wait for it before reading)
    import torch
    od = to_device(np.zeros_like(out))
    m.mglma_contract(ctx, L, nrhs, to_device(a), to_device(b), od)
    torch.cuda.synchronize()
    assert np.array_equal(od.cpu().numpy(), out)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_gamma5_gamma_bit_exact(m, ctx, k):
    L = (4, 2, 3, 2)
    psi = synthetic.random_spinors(L, 2, 83)
    out = np.zeros_like(psi)
    m.mglma_gamma5_gamma(ctx, L, k, 2, psi, out)
    assert np.array_equal(out, K.spin_apply(K.gamma5_gamma(k), psi))
    with pytest.raises(m.MglmaError):
        m.mglma_gamma5_gamma(ctx, L, 4, 2, psi, out)


def test_estimator_equals_trace_formula(m, ctx):
    """Exact dilution of slice y0 (12 point sources per site), each source and
    its gamma5 gamma_k images solved in FP64 on the GPU, contracted on the
    GPU: the sum equals C(x0, y0) of Eq. tmr from the dense inverse."""
    L, y0, kappa, csw = (4, 2, 2, 2), 1, 0.125, 1.3
    V = int(np.prod(L))
    U = synthetic.gauge_links(L, 0.4, 5)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    slice_ = V // L[0]
    n = slice_ * 12
    sites = [y0 * slice_ + s for s in range(slice_) for _ in range(12)]
    cols = [e for _ in range(slice_) for e in range(12)]
    eta = np.zeros((n,) + L + (4, 3), dtype=np.complex128)
    m.mglma_sources(ctx, L, m.MGLMA_SOURCE_POINT, n, 0, eta, point_sites=sites, point_sc=cols)
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_CGNE, tol=1e-12)
    b = np.zeros_like(eta)
    m.mglma_solve_batch(ctx, g, None, prm, [n], eta, b)
    a = np.zeros((n, 3) + L + (4, 3), dtype=np.complex128)
    for k in (1, 2, 3):
        src = np.zeros_like(eta)
        m.mglma_gamma5_gamma(ctx, L, k, n, eta, src)
        x = np.zeros_like(eta)
        m.mglma_solve_batch(ctx, g, None, prm, [n], src, x)
        a[:, k - 1] = x
    out = np.zeros((n, L[0]), dtype=np.complex128)
    m.mglma_contract(ctx, L, n, a, b, out)
    C = K.correlator_from_propagator(np.linalg.inv(D.dense_dirac(U, kappa, csw)), L, y0)
    assert np.abs(out.sum(axis=0) - C).max() <= 1e-9 * np.abs(C).max()
    m.mglma_gauge_free(g)
