"""Serving with continuous batching: requests that arrive while others run
share the slots and kernel launches; each result equals the solve of that
request alone (within the solver tolerance) and reaches the FP64 residual
target as computed by the oracle; latency statistics are reported."""
import numpy as np
import pytest

import synthetic
from oracle import dirac as D
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


def make_lattice(m, ctx, L, b, nv, eps, seed, kappa, csw):
    U = synthetic.gauge_links(L, eps, seed)
    g = m.mglma_gauge_load(ctx, L, U, kappa, csw)
    sub = m.mglma_subspace_create(ctx, g, b, nv, 5, seed + 1, m.MGLMA_FP32, n_cg=20, cg_prec=m.MGLMA_FP32)
    C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
    return dict(L=L, U=U, g=g, sub=sub, C=C, kappa=kappa, csw=csw)


def test_serve_mix_equals_alone(m, ctx):
    A = make_lattice(m, ctx, (8, 8, 8, 8), (2, 2, 2, 2), 8, 0.3, 1001, 0.12, 1.0)
    B = make_lattice(m, ctx, (8, 4, 4, 8), (2, 2, 2, 2), 4, 0.2, 1011, 0.125, 1.7)
    lats = [A, B]
    spec = [(0, 2, 0.0), (1, 1, 0.0), (0, 3, 0.005), (0, 1, 0.01), (1, 2, 0.02), (0, 4, 0.03)]
    reqs = []
    for i, (l, n, t) in enumerate(spec):
        b = synthetic.z2_noise(lats[l]["L"], n, 5000 + i)
        reqs.append(dict(lattice=l, b=b, x=np.zeros_like(b), arrival=t))
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG)
    stats, res = m.mglma_serve(ctx, [(A["g"], A["C"]), (B["g"], B["C"])], reqs, prm, max_slots=3)
    assert stats["requests"] == len(spec) and stats["rejected"] == 0
    assert stats["rhs"] == sum(n for _, n, _ in spec)
    assert stats["slots"] == [3, 3] and 0 < stats["p50_s"] <= stats["p99_s"] <= stats["max_s"]
    for i, r in enumerate(reqs):
        assert res[i]["status"] == 0 and all(s["converged"] for s in res[i]["stats"])
        lt = lats[r["lattice"]]
        # alone: the same sources through the batch solver
        xa = np.zeros_like(r["b"])
        m.mglma_solve_batch(ctx, lt["g"], lt["C"], prm, [r["b"].shape[0]], r["b"], xa)
        for j in range(r["b"].shape[0]):
            assert np.linalg.norm(r["x"][j] - xa[j]) <= 1e-9 * np.linalg.norm(xa[j])
            assert S.true_residual(lt["U"], r["x"][j], r["b"][j], lt["kappa"], lt["csw"]) <= 1e-10
    for lt in lats:
        m.mglma_coarse_free(lt["C"])
        m.mglma_subspace_free(lt["sub"])
        m.mglma_gauge_free(lt["g"])


def test_serve_device_buffers_and_request_larger_than_slots(m, ctx):
    import torch
    A = make_lattice(m, ctx, (4, 4, 4, 8), (2, 2, 2, 2), 4, 0.3, 1021, 0.12, 1.0)
    b = torch.from_numpy(synthetic.z2_noise(A["L"], 5, 5100)).cuda()
    x = torch.zeros_like(b)
    reqs = [dict(lattice=0, b=b, x=x, arrival=0.0),
            dict(lattice=7, b=b, x=x, arrival=0.0)]  # unknown lattice -> invalid
    stats, res = m.mglma_serve(ctx, [(A["g"], A["C"])], reqs, max_slots=2)
    assert res[0]["status"] == 0 and res[1]["status"] == 1 and stats["rejected"] == 1
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    for j in range(5):
        assert S.true_residual(A["U"], xh[j], bh[j], A["kappa"], A["csw"]) <= 1e-10
    m.mglma_coarse_free(A["C"])
    m.mglma_subspace_free(A["sub"])
    m.mglma_gauge_free(A["g"])


def test_serve_lean_device_generated_lattices(m, ctx):
    """The serving set-up used for the large boxes, on small lattices: links
    generated on the device, lean FP16 basis (test vectors relaxed in groups,
    no FP64 copy), BF16 coarse operator with its FP64 copy released, slots
    sized by volume share.  Every result reaches 1e-10 in the oracle's FP64
    residual (computed with the host generator's links) and equals the solve
    of the same sources alone."""
    spec_l = [((8, 8, 8, 8), 0.15, 1051), ((8, 4, 4, 8), 0.2, 1052)]
    kappa, csw = 0.125, 1.7
    lats = []
    for L, eps, seed in spec_l:
        g = m.mglma_gauge_random(ctx, L, eps, seed, kappa, csw)
        sub = m.mglma_subspace_create(ctx, g, (2, 2, 2, 2), 6, 5, seed + 1, m.MGLMA_FP16, n_cg=20,
                                      cg_prec=m.MGLMA_FP32, lean_group=4)
        C = m.mglma_coarse_build(ctx, g, sub, m.MGLMA_BF16)
        m.mglma_coarse_release_fp64(C)
        lats.append(dict(L=L, U=synthetic.gauge_links(L, eps, seed), g=g, sub=sub, C=C))
    spec = [(0, 1, 0.0), (1, 2, 0.0), (0, 2, 0.01), (1, 1, 0.02), (0, 1, 0.03)]
    reqs = []
    for i, (l, n, t) in enumerate(spec):
        b = synthetic.z2_noise(lats[l]["L"], n, 5200 + i)
        reqs.append(dict(lattice=l, b=b, x=np.zeros_like(b), arrival=t))
    prm = m.mglma_solve_params_default(m.MGLMA_SOLVER_MG)
    stats, res = m.mglma_serve(ctx, [(lt["g"], lt["C"]) for lt in lats], reqs, prm, max_slots=2, hbm_fraction=0.5)
    assert stats["rejected"] == 0 and stats["rhs"] == sum(n for _, n, _ in spec)
    for i, r in enumerate(reqs):
        assert res[i]["status"] == 0
        lt = lats[r["lattice"]]
        xa = np.zeros_like(r["b"])
        m.mglma_solve_batch(ctx, lt["g"], lt["C"], prm, [r["b"].shape[0]], r["b"], xa)
        for j in range(r["b"].shape[0]):
            assert np.linalg.norm(r["x"][j] - xa[j]) <= 1e-9 * np.linalg.norm(xa[j])
            assert S.true_residual(lt["U"], r["x"][j], r["b"][j], kappa, csw) <= 1e-10
    for lt in lats:
        m.mglma_coarse_free(lt["C"])
        m.mglma_subspace_free(lt["sub"])
        m.mglma_gauge_free(lt["g"])
