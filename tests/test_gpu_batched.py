"""Batched solve: every problem's result equals its own solve and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2107_11810_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11810_gb300 import build
    build.build()


@pytest.mark.parametrize("workers", [1, 3])
def test_batched_equals_single_solves_and_oracle(workers):
    from paper_2107_11810_gb300 import vote
    probs = inputs.pose3dof_batch(num=12, n_lo=1, n_hi=3000, seed=51)
    probs.insert(3, inputs.pose3dof(n=0, seed=52))             # an empty problem in the middle
    p0 = probs[0]
    s = vote.Solver(p0.family, p0.eps, p0.bounds)
    s.set_option(vote.VOTE_OPT_BATCH_WORKERS, workers)
    flat, offs = vote.pack_batch([p.params for p in probs])
    res = s.solve_batched((torch.from_numpy(flat).cuda(), offs))
    masks = vote.mask_words_to_numpy(res["masks"])
    for b, p in enumerate(probs):
        o = oracle.solve(p.family, p.eps, p.bounds, p.params)
        assert res["depths"][b] == o["depth"]
        assert np.array_equal(res["best_leaves"][b], o["best_leaf"])
        assert np.array_equal(res["best_points"][b], o["best_point"])
        w0, nw = res["word_offsets"][b], (p.n + 31) // 32
        assert np.array_equal(masks[w0:w0 + nw], o["mask"])
    assert np.all(res["latency_ms"] > 0)
    # the batch's counters are the totals of the problems' own solves
    s1 = vote.Solver(p0.family, p0.eps, p0.bounds)
    tests = launches = 0
    for p in probs:
        s1.solve(torch.from_numpy(np.ascontiguousarray(p.params)).cuda())
        tests += s1.stats()["tests"]
        launches += s1.stats()["launches"]
    st = s.stats()
    assert st["tests"] == tests and st["launches"] == launches > 0


def test_batched_rejects_bad_offsets():
    from paper_2107_11810_gb300 import vote
    p = inputs.pose3dof(n=100, seed=53)
    s = vote.Solver(p.family, p.eps, p.bounds)
    flat = torch.from_numpy(p.params.ravel().copy()).cuda()
    with pytest.raises(vote.VoteError):
        s.solve_batched((flat, np.array([0, 60, 40, 100])))
