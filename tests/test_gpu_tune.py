"""The launch-shape autotuner (mcs_options.tune, tune_cache): it times the candidate shapes of the batched
facet step (2D) and of the staged K apply on the handle's own data, keeps the fastest, and records them
in a cache file that later handles of the same (dim, k, precision, element count) read instead of
tuning.  Shapes change only the grouping of facets and elements into blocks, never the arithmetic of
one facet or element, so results are bitwise those of the formula shapes."""
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


@pytest.mark.parametrize("d,N,k,prec", [(2, 16, 3, "mixed"), (2, 8, 2, "fp64"), (3, 4, 2, "mixed")])
def test_tuned_shapes_give_the_same_results(mcs, tmp_path, d, N, k, prec):
    p = mcs.MCS_MIXED if prec == "mixed" else mcs.MCS_FP64
    cache = str(tmp_path / "tune.txt")
    ref = mcs.Handle.structured(d, N, k, 1.0, precision=p)
    ref.condense()
    h = mcs.Handle.structured(d, N, k, 1.0, precision=p, tune=1, tune_cache=cache)
    h.condense()
    s = h.sizes
    assert s.apply_batch > 0
    if d == 2:
        assert s.facet_batch > 0 and s.facet_threads in (128, 256)
    rng = np.random.default_rng(4)
    r = torch.tensor(rng.standard_normal(s.ndof), device="cuda")
    outs = []
    for hh in (ref, h):
        z = torch.zeros_like(r)
        y = torch.zeros_like(r)
        hh.precond(r, z)
        hh.apply(r, y)
        torch.cuda.synchronize()
        outs.append((z.cpu().numpy(), y.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    # the K apply sums two element contributions per facet dof with atomics: equal to the last bit
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-15 * np.abs(outs[0][1]).max()
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith(f"mcs-tune dim={d} k={k}")
    # a second handle takes the cached shapes without timing (the file keeps one line)
    h2 = mcs.Handle.structured(d, N, k, 1.0, precision=p, tune=1, tune_cache=cache)
    h2.condense()
    s2 = h2.sizes
    assert (s2.facet_batch, s2.facet_threads, s2.apply_batch) == (s.facet_batch, s.facet_threads, s.apply_batch)
    assert len(open(cache).read().splitlines()) == 1
    for hh in (ref, h, h2):
        hh.close()
