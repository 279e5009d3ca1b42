"""The allocation-free Dirac apply (mglma_dirac_apply_noalloc) against the
regular mglma_dirac_apply, through the C ABI.

Some callers cannot allocate device memory when they need the operator (for
example code running inside a CUDA graph capture, or a process whose HBM is
already held by another caching allocator); the no-alloc entry point keeps
its work fields in a fixed 32 MiB device array instead.  Two calls in a row
must each give the regular entry point's result, and requests beyond the
array or with host buffers must be refused.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes alone."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2412_06347_gb300 as m
    ctx = m.Context(0)
    L = (8, 8, 8, 8)
    U = synthetic.gauge_links(L, 0.3, 1001)
    g = m.mglma_gauge_load(ctx, L, U, 0.12, 1.0)
    yield m, torch, ctx, g, L
    m.mglma_gauge_free(g)
    ctx.close()


@pytest.mark.parametrize("op", [0, 1, 2, 3])
@pytest.mark.parametrize("compute,tol", [(0, 1e-12), (1, 2e-6)])
def test_noalloc_matches_regular_two_calls(env, op, compute, tol):
    m, torch, ctx, g, L = env
    for call, seed in enumerate((5, 6)):  # two calls in a row share the array
        nrhs = 3 if call == 0 else 2
        psi = torch.from_numpy(synthetic.random_spinors(L, nrhs, seed)).cuda()
        ref = torch.zeros_like(psi)
        got = torch.full_like(psi, float("nan"))
        # both calls run on torch's current stream, after the fills above
        stream = torch.cuda.current_stream().cuda_stream
        m.mglma_dirac_apply(ctx, g, op, nrhs, psi, ref, compute, stream=stream)
        m.mglma_dirac_apply_noalloc(ctx, g, op, nrhs, psi, got, compute, stream=stream)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), got.cpu().numpy()
        err = np.linalg.norm((o - r).reshape(nrhs, -1), axis=1) / np.linalg.norm(r.reshape(nrhs, -1), axis=1)
        assert err.max() <= tol, (call, err)


def test_noalloc_rejects_oversize_and_host_buffers(env):
    m, torch, ctx, g, L = env
    V = int(np.prod(L))
    nrhs = 87381 // V + 1  # FP64: two fields of nrhs x V x 192 bytes exceed 32 MiB
    big = torch.zeros((nrhs, V, 12), dtype=torch.complex128, device="cuda")
    with pytest.raises(m.MglmaError) as e:
        m.mglma_dirac_apply_noalloc(ctx, g, 0, nrhs, big, big, m.MGLMA_FP64)
    assert e.value.status == 1 and "scratch" in str(e.value)
    host = synthetic.random_spinors(L, 1, 7)
    with pytest.raises(m.MglmaError) as e:
        m.mglma_dirac_apply_noalloc(ctx, g, 0, 1, host, np.zeros_like(host), m.MGLMA_FP64)
    assert e.value.status == 1
