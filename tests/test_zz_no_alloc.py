"""mcs_condense_noalloc: element matrices for callers that cannot allocate device memory.

Applications that own the whole device through their own memory pool or run under a hard memory
budget, and code paths that must not block on the allocator, need an entry point that allocates
nothing.  This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def mcs():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as m
    return m


@pytest.mark.parametrize("d,N,k,nu", [(2, 8, 3, 0.7), (3, 2, 2, 1.3), (3, 1, 4, 0.5), (3, 2, 1, 1.0)])
def test_noalloc_condense_matches_condense(mcs, d, N, k, nu):
    """Two calls in a row of the no-allocation entry point against mcs_condense's A_T."""
    h = mcs.Handle.structured(d, N, k, nu, precision=mcs.MCS_FP64, gmg_levels=1)
    h.condense()
    s = h.sizes
    ref = h.element_matrices(0, s.ne)                  # packed lower triangles from mcs_condense
    il = np.tril_indices(s.n_A)
    for T0, count in [(0, s.ne), (s.ne // 3, s.ne - s.ne // 3)]:
        out = torch.full((count, s.n_A, s.n_A), float("nan"), dtype=torch.float64, device="cuda")
        h.condense_noalloc(T0, count, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()[:, il[0], il[1]]
        want = ref[T0:T0 + count]
        err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
        assert np.isfinite(got).all() and err.max() < 1e-12, err.max()
        assert np.abs(out.cpu().numpy() - np.transpose(out.cpu().numpy(), (0, 2, 1))).max() == 0.0
    h.close()


def test_noalloc_rejects_bad_arguments(mcs):
    h = mcs.Handle.structured(2, 4, 2, 1.0, precision=mcs.MCS_FP64, gmg_levels=1)
    out = torch.zeros((1, h.sizes.n_A, h.sizes.n_A), dtype=torch.float64, device="cuda")
    with pytest.raises(mcs.McsError) as e:
        h.condense_noalloc(h.sizes.ne, 1, out)
    assert e.value.code == mcs.MCS_ERR_INVALID_ARG
    # buffers the kernel would overrun are refused by the binding before any launch
    with pytest.raises(ValueError):
        h.condense_noalloc(0, 2, out)                              # one element's room for two
    with pytest.raises(ValueError):
        h.condense_noalloc(0, 1, out.to(torch.float32))
    h.close()
