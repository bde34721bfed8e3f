"""Parity of the CUDA path with the oracle for the radial camera (RADIAL5DOF,
Sec. 4.2.4: 5 coordinates, 32 children per cell through the wide kernels), through
the C ABI.

Depth, best leaf, best point and inlier mask must be bit-exact in both precision
modes; the per-cell UB/LB trace of an unpruned search equals the oracle's; with
grouping and with small expansion steps the results do not change; replayed cell
counts equal the oracle's.
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


def vote_mod():
    from paper_2107_11810_gb300 import vote
    return vote


def gpu_solve(p, precision=1, params=None, **kw):
    v = vote_mod()
    opts = {k: kw.pop(k) for k in list(kw) if k.startswith("VOTE_OPT_")}
    s = v.Solver(p.family, p.eps, p.bounds, precision=precision, **kw)
    for k, val in opts.items():
        s.set_option(getattr(v, k), val)
    x = p.params if params is None else params
    r = s.solve(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    r["mask"] = v.mask_words_to_numpy(r["mask"])
    r["solver"] = s
    return r


def assert_same(g, o, n):
    assert g["depth"] == o["depth"]
    assert np.array_equal(g["best_leaf"], o["best_leaf"])
    assert np.array_equal(g["best_point"], o["best_point"])
    assert np.array_equal(g["mask"][: (n + 31) // 32], o["mask"])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,levels,seed", [(1, 3, 1), (40, 3, 2), (300, 4, 3)])
def test_small_parity(precision, n, levels, seed):
    p = inputs.radial5dof(n=n, inlier_frac=0.3, levels=levels, seed=seed)
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    g = gpu_solve(p, precision)
    assert_same(g, o, p.n)
    assert int(np.unpackbits(g["mask"].view(np.uint8)).sum()) == g["depth"]


def test_full_trace_without_pruning_equals_oracle():
    p = inputs.radial5dof(n=60, inlier_frac=0.3, levels=3, seed=5)
    cap = 4_000_000
    o = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=oracle.NO_PRUNE, trace_cap=cap)
    g = gpu_solve(p, 1, prune=False, trace_cap=cap)
    tg = g["solver"].trace(cap)
    to = o["trace"]
    key = lambda l, c: (int(l), tuple(int(x) for x in c))
    dg = {key(l, c): (int(u), int(b)) for l, c, u, b in zip(tg["level"], tg["coords"], tg["ub"], tg["lb"])}
    do = {key(l, c): (int(u), int(b)) for l, c, u, b in zip(to["level"], to["coords"], to["ub"], to["lb"])}
    assert len(tg["level"]) == len(dg)
    assert dg == do
    assert_same(g, o, p.n)


@pytest.mark.parametrize("precision", [0, 1])
def test_grouping_and_small_steps_do_not_change_results(precision):
    p = inputs.radial5dof(n=200, inlier_frac=0.3, levels=4, seed=6)
    params = np.concatenate([p.params, p.params[:, :60]], axis=1)      # repeats merge
    o = oracle.solve(p.family, p.eps, p.bounds, params)
    g = gpu_solve(p, precision, params=params, VOTE_OPT_GROUP=1)
    assert_same(g, o, params.shape[1])
    g = gpu_solve(p, precision, params=params, chunk_records=500)
    assert_same(g, o, params.shape[1])


def test_cell_counts_replay_equals_oracle():
    p = inputs.radial5dof(n=300, inlier_frac=0.3, levels=4, seed=7)
    v = vote_mod()
    s = v.Solver(p.family, p.eps, p.bounds)
    t = torch.from_numpy(p.params).cuda()
    rng = np.random.default_rng(3)
    for level in (0, 1, 2, 4):
        for _ in range(3):
            coords = [int(rng.integers(0, 2 ** level)) for _ in range(p.d)]
            ub, lb, reach = s.cell_counts(t, level, coords, want_reach=True)
            oub, olb, oreach = oracle.cell_counts(p.family, p.eps, p.bounds, p.params, level, coords, want_reach=True)
            assert (ub, lb) == (oub, olb)
            assert np.array_equal(v.mask_words_to_numpy(reach), oreach)
