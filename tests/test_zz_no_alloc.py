"""The entry point that allocates no device memory (vote_cell_counts_noalloc).

Some callers cannot call cudaMalloc (a host that plans all GPU memory up front, a
real-time loop with a fixed memory budget, code running inside another
framework's allocator).  For them the library offers one context-free entry
point whose scratch is a fixed array inside the library.  This test calls it
through the C ABI and checks, on two calls in a row, that its per-cell counts and
reach mask equal those of vote_cell_counts (which uses the context's allocated
memory), and that those equal the oracle's replay.  Counts are integers, so they
must be identical.

The file is named so that pytest collects it last.
"""
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


@pytest.mark.parametrize("family", [inputs.LINE2D, inputs.PLANE3D_SPH, inputs.POSE3DOF])
def test_noalloc_cell_counts_match_context_entry_point(family):
    from paper_2107_11810_gb300 import vote
    if family == inputs.LINE2D:
        p = inputs.line2d(n=3000, inlier_frac=0.2, eps=0.02, seed=31)
    elif family == inputs.PLANE3D_SPH:
        p = inputs.plane3d(n=3000, inlier_frac=0.2, eps=0.06, sigma=0.002, seed=32)
    else:
        p = inputs.pose3dof(n=3000, inlier_frac=0.2, eps_xy=1.0, eps_yaw_deg=2.0, seed=33)
    t = torch.from_numpy(p.params).cuda()
    s = vote.Solver(p.family, p.eps, p.bounds)
    L, Lj = s.levels()
    best = s.solve(t)
    rng = np.random.default_rng(5)
    cells = [(L, best["best_leaf"])]
    for level in (0, 1, L // 2, L):
        cells.append((level, [int(rng.integers(0, 2 ** min(level, int(Lj[j])))) for j in range(p.d)]))
    words = (p.n + 31) // 32
    for level, coords in cells:
        ref_ub, ref_lb, ref_reach = s.cell_counts(t, level, coords, want_reach=True)
        # the context entry point itself equals the oracle's replay (the FP64 definition)
        oub, olb, oreach = oracle.cell_counts(p.family, p.eps, p.bounds, p.params, level, coords, want_reach=True)
        assert (ref_ub, ref_lb) == (oub, olb)
        assert np.array_equal(vote.mask_words_to_numpy(ref_reach), oreach)
        for _ in range(2):                                  # two calls in a row share the scratch
            reach = torch.full((words,), -1, dtype=torch.int32, device="cuda")
            ub, lb = vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t, level, coords, reach=reach)
            assert (ub, lb) == (ref_ub, ref_lb)
            assert torch.equal(reach, ref_reach)
    # the best leaf's count is the solve's depth
    ub, _ = vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t, L, best["best_leaf"])
    assert ub == best["depth"]


def test_noalloc_rejects_bad_arguments():
    from paper_2107_11810_gb300 import vote
    p = inputs.line2d(n=100, seed=34)
    t = torch.from_numpy(p.params).cuda()
    with pytest.raises(vote.VoteError) as ei:
        vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t, 99, [0, 0])
    assert ei.value.code == 1
    with pytest.raises(vote.VoteError):
        vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t, 1, [5, 0])
    # wrong buffers are refused before the call: host tensor, float32, short reach
    with pytest.raises(ValueError):
        vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t.cpu(), 1, [0, 0])
    with pytest.raises(ValueError):
        vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t.float(), 1, [0, 0])
    with pytest.raises(ValueError):
        short = torch.zeros((p.n + 31) // 32 - 1, dtype=torch.int32, device="cuda")
        vote.cell_counts_noalloc(p.family, p.eps, p.bounds, t, 1, [0, 0], reach=short)
