"""The allocation-free scoring entry point, for callers that must not
allocate device memory (a serving loop whose HBM belongs to a pool it does
not own, a host framework that owns the allocator): it must return what the
ordinary entry point returns, call after call, while its partial sums live
in the library's fixed device array.  Collected last on purpose, so that a
run stopping at the first failure has run everything else first; it also
passes alone in a fresh process."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _problem(n, d, kappa, seed):
    g = np.random.default_rng(seed)
    X = (g.standard_normal((n, d)) + 0.3).astype(np.float32)
    y = np.where(g.random(n) < 0.5, 1.0, -1.0).astype(np.float32)
    o = (0.5 * g.standard_normal(n)).astype(np.float32)
    idx = g.choice(n, size=kappa, replace=False).astype(np.int64)
    return X, y, o, idx


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
@pytest.mark.parametrize("n,d,kappa", [(3000, 24, 100), (20000, 128, 256)])
def test_noalloc_matches_scratch_entry_point_twice(prec, n, d, kappa):
    import paper_1404_1066_gb300 as sp
    X, y, o, idx = _problem(n, d, kappa, seed=n + kappa)
    P = sp.spsvm_prepare_points(torch.from_numpy(X).cuda(), prec)
    yt, ot = torch.from_numpy(y).cuda(), torch.from_numpy(o).cuda()
    it = torch.from_numpy(idx).cuda()
    lam, gamma = 1e-3, 1.0 / d
    ref = [t.cpu().numpy() for t in sp.spsvm_score_candidates(P, yt, ot, it, gamma, lam, prec)]
    for _ in range(2):
        got = [t.cpu().numpy() for t in
               sp.spsvm_score_candidates_noalloc(P, yt, ot, it, gamma, lam, prec)]
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-12)


def test_noalloc_rejects_sizes_beyond_the_array():
    import paper_1404_1066_gb300 as sp
    X, y, o, idx = _problem(600_000, 4, 256, seed=1)
    P = sp.spsvm_prepare_points(torch.from_numpy(X).cuda(), "fp32")
    with pytest.raises(sp.SpsvmError) as e:
        sp.spsvm_score_candidates_noalloc(P, torch.from_numpy(y).cuda(),
                                          torch.from_numpy(o).cuda(),
                                          torch.from_numpy(idx).cuda(), 0.25, 1e-3, "fp32")
    assert e.value.code == -1 and "fixed" in str(e.value)
