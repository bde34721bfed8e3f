"""Autotuner: cache keying and selection (CPU, with a fake timer and solver), and
on the GPU that every candidate setting gives the same result."""
import numpy as np
import pytest

from paper_2107_11810_gb300 import autotune, inputs


class FakeSolver:
    family, d = 2, 3

    def __init__(self):
        self.opts = {}

    def set_option(self, k, v):
        self.opts[k] = v


class FakeSurfaces:
    shape = (3, 12345)


def test_buckets_and_keys():
    assert autotune.n_bucket(1) == 0
    assert autotune.n_bucket(4 ** 5) == 5
    assert autotune.n_bucket(4 ** 5 + 1) == 5
    assert autotune.cache_key(2, 3, 10 ** 6, "GB300") == "2:3:9:GB300"


def test_tune_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    s = FakeSolver()
    cost = {1 << 23: 3.0, 1 << 25: 1.0, 1 << 26: 2.0, 1 << 27: 2.5}

    def timer(solver, x):
        return cost[solver.opts[3]]

    out = autotune.tune(s, FakeSurfaces(), timer=timer, gpu="GB300", cache_path=path)
    assert out["best"] == dict(chunk_records=1 << 25)
    assert s.opts[3] == 1 << 25
    s2 = FakeSolver()
    assert autotune.apply_cached(s2, 12000, "GB300", cache_path=path)
    assert s2.opts[3] == 1 << 25
    assert not autotune.apply_cached(s2, 12, "GB300", cache_path=path)


@pytest.mark.gpu
def test_every_candidate_gives_the_same_result():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11810_gb300 import build, vote
    build.build()
    p = inputs.plane3d(n=20000, inlier_frac=0.05, eps=0.02, seed=71)
    s = vote.Solver(p.family, p.eps, p.bounds)
    t = torch.from_numpy(p.params).cuda()
    ref = s.solve(t)
    out = autotune.tune(s, t, cache_path=None)
    for c, _ in out["times"]:
        autotune.apply(s, c)
        r = s.solve(t)
        assert r["depth"] == ref["depth"] and np.array_equal(r["best_leaf"], ref["best_leaf"])
        assert torch.equal(r["mask"], ref["mask"])
