"""Parity of the CUDA path with the oracle, through the C ABI.

Counts, depth, best leaf and inlier mask are integer results decided by FP64
comparisons and must be bit-exact, in both precision modes (plain FP64 predicate
and FP32 screen with FP64 recheck).  The best point is the leaf centre computed
by the same formula on both sides; it is compared exactly as well.
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


def dev(p):
    return torch.from_numpy(np.ascontiguousarray(p.params)).cuda()


def gpu_solve(p, precision=1, **kw):
    v = vote_mod()
    s = v.Solver(p.family, p.eps, p.bounds, precision=precision, **kw)
    r = s.solve(dev(p))
    r["mask"] = v.mask_words_to_numpy(r["mask"])
    r["stats"] = s.stats()
    r["solver"] = s
    return r


def assert_same(g, o, n):
    assert g["depth"] == o["depth"]
    assert np.array_equal(g["best_leaf"], o["best_leaf"])
    assert np.array_equal(g["best_point"], o["best_point"])
    assert np.array_equal(g["mask"][: (n + 31) // 32], o["mask"])


def small(family, n, seed):
    if family == inputs.LINE2D:
        return inputs.line2d(n=n, inlier_frac=0.2, eps=0.02, seed=seed)
    if family == inputs.PLANE3D_SPH:
        return inputs.plane3d(n=n, inlier_frac=0.2, eps=0.06, sigma=0.002, seed=seed)
    if family == inputs.RAYS3D:
        return inputs.rays3d(n=n, inlier_frac=0.2, eps=0.02, noise=0.002, seed=seed)
    if family == inputs.AFFINE4D:
        return inputs.affine4d(n=n, inlier_frac=0.3, eps=0.1, noise=0.005, seed=seed)
    if family == inputs.POINTSET2D:          # n ~ m^2 correspondences
        return inputs.pointset2d(m=max(1, int(round(n ** 0.5))), eps=0.05, noise=0.002, seed=seed)
    return inputs.pose3dof(n=n, inlier_frac=0.2, eps_xy=1.0, eps_yaw_deg=2.0, noise_deg=0.05, seed=seed)


FAMS = [inputs.LINE2D, inputs.PLANE3D_SPH, inputs.POSE3DOF, inputs.RAYS3D, inputs.POINTSET2D, inputs.AFFINE4D]


@pytest.mark.parametrize("family", FAMS)
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,seed", [(1, 1), (33, 2), (517, 3), (2000, 4)])
def test_small_parity(family, precision, n, seed):
    p = small(family, n, seed)
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    g = gpu_solve(p, precision)
    assert_same(g, o, p.n)
    assert int(np.unpackbits(g["mask"].view(np.uint8)).sum()) == g["depth"]


def test_line2d_workload_parity_both_modes():
    p = inputs.line2d()                         # 10,000 points, eps = 0.01
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    for prec in (0, 1):
        g = gpu_solve(p, prec)
        assert_same(g, o, p.n)


def test_pose3dof_1e5_parity():
    p = inputs.pose3dof(n=100_000, seed=inputs.SEED_BASE + 2)
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    g = gpu_solve(p, 1)
    assert_same(g, o, p.n)


def test_plane3d_parity_several_tiles():
    p = inputs.plane3d(n=3000, inlier_frac=0.05, eps=0.03, sigma=0.002, seed=9)
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    g1 = gpu_solve(p, 1)
    g0 = gpu_solve(p, 0)
    assert_same(g1, o, p.n)
    assert_same(g0, o, p.n)
    assert g1["stats"]["tests"] > 0


@pytest.mark.parametrize("family", FAMS)
def test_full_trace_without_pruning_equals_oracle(family):
    p = small(family, 300 if family != inputs.PLANE3D_SPH else 60, 5)
    if family == inputs.POINTSET2D:          # 16 children per cell: fewer levels keep the trace small
        p = inputs.pointset2d(m=10, eps=0.2, noise=0.002, seed=5)
    if family == inputs.AFFINE4D:
        p = inputs.affine4d(n=60, inlier_frac=0.3, eps=0.3, noise=0.005, seed=5)
    cap = 4_000_000
    o = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=oracle.NO_PRUNE, trace_cap=cap)
    g = gpu_solve(p, 1, prune=False, trace_cap=cap)
    tg = g["solver"].trace(cap)
    to = o["trace"]
    key = lambda l, c: (int(l), tuple(int(x) for x in c))
    dg = {key(l, c): (int(u), int(b)) for l, c, u, b in zip(tg["level"], tg["coords"], tg["ub"], tg["lb"])}
    do = {key(l, c): (int(u), int(b)) for l, c, u, b in zip(to["level"], to["coords"], to["ub"], to["lb"])}
    assert len(tg["level"]) == len(dg)          # no cell tested twice (the dive's cells included)
    assert dg == do
    assert_same(g, o, p.n)


@pytest.mark.parametrize("family", FAMS)
def test_pruned_trace_entries_equal_oracle_cell_counts(family):
    p = small(family, 1500, 6)
    g = gpu_solve(p, 1, trace_cap=4_000_000)
    tg = g["solver"].trace(4_000_000)
    rng = np.random.default_rng(1)
    for x in rng.choice(len(tg["ub"]), size=min(30, len(tg["ub"])), replace=False):
        ub, lb = oracle.cell_counts(p.family, p.eps, p.bounds, p.params, tg["level"][x], tg["coords"][x])
        assert (ub, lb) == (tg["ub"][x], tg["lb"][x])


@pytest.mark.parametrize("family", FAMS)
def test_cell_counts_replay_equals_oracle(family):
    p = small(family, 2500, 7)
    v = vote_mod()
    s = v.Solver(p.family, p.eps, p.bounds)
    t = dev(p)
    L, Lj = s.levels()
    rng = np.random.default_rng(3)
    for level in sorted(set([0, 1, L // 2, L])):
        for _ in range(3):
            coords = [int(rng.integers(0, 2 ** min(level, int(Lj[j])))) for j in range(p.d)]
            ub, lb, reach = s.cell_counts(t, level, coords, want_reach=True)
            oub, olb, oreach = oracle.cell_counts(p.family, p.eps, p.bounds, p.params, level, coords, want_reach=True)
            assert (ub, lb) == (oub, olb)
            assert np.array_equal(v.mask_words_to_numpy(reach), oreach)


@pytest.mark.parametrize("family", FAMS)
@pytest.mark.parametrize("precision", [0, 1])
def test_grouping_parity_and_merging(family, precision):
    # grouping merges equal canonical records; results must not change
    v = vote_mod()
    p = small(family, 2500, 15)
    params = np.concatenate([p.params, p.params[:, :700], p.params[:, :300]], axis=1)   # duplicates merge
    o = oracle.solve(p.family, p.eps, p.bounds, params)
    s0 = v.Solver(p.family, p.eps, p.bounds, precision=precision, chunk_records=4000)
    s1 = v.Solver(p.family, p.eps, p.bounds, precision=precision, chunk_records=4000)
    s1.set_option(v.VOTE_OPT_GROUP, 1)
    t = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    r0, r1 = s0.solve(t), s1.solve(t)
    for r in (r0, r1):
        r["mask"] = v.mask_words_to_numpy(r["mask"])
        assert_same(r, o, params.shape[1])
    assert s1.stats()["records"] < s0.stats()["records"]
    assert s1.stats()["tests"] < s0.stats()["tests"]


@pytest.mark.parametrize("chunk", [1, 2, 7, 1000])
@pytest.mark.parametrize("dive", [0, 1])
def test_chunking_and_dive_do_not_change_results(chunk, dive):
    v = vote_mod()
    for fam in FAMS:
        p = small(fam, 3000, 8)
        o = oracle.solve(p.family, p.eps, p.bounds, p.params)
        s = v.Solver(p.family, p.eps, p.bounds, chunk_records=chunk)
        s.set_option(v.VOTE_OPT_DIVE, dive)
        g = s.solve(dev(p))
        g["mask"] = v.mask_words_to_numpy(g["mask"])
        assert_same(g, o, p.n)


def test_empty_and_degenerate_inputs():
    v = vote_mod()
    p = small(inputs.LINE2D, 50, 9)
    s = v.Solver(p.family, p.eps, p.bounds)
    r = s.solve(torch.zeros((2, 0), dtype=torch.float64, device="cuda"))
    assert r["depth"] == 0 and np.all(r["best_leaf"] == 0)
    same = np.repeat(p.params[:, :1], 77, axis=1)
    r = s.solve(torch.from_numpy(same).cuda())
    o = oracle.solve(p.family, p.eps, p.bounds, same)
    assert r["depth"] == o["depth"] == 77
    assert np.array_equal(r["best_leaf"], o["best_leaf"])
    # eps covering the whole domain: the root is the only leaf
    s2 = v.Solver(p.family, [5.0, 5.0], p.bounds)
    r = s2.solve(dev(p))
    assert r["depth"] == p.n
    assert np.all(v.mask_words_to_numpy(r["mask"])[: p.n // 32] == 0xFFFFFFFF)


def test_invalid_inputs_return_einval_and_context_survives():
    v = vote_mod()
    p = small(inputs.LINE2D, 100, 10)
    s = v.Solver(p.family, p.eps, p.bounds)
    bad = p.params.copy()
    bad[1, 17] = np.inf
    with pytest.raises(v.VoteError) as ei:
        s.solve(torch.from_numpy(bad).cuda())
    assert ei.value.code == 1
    huge = p.params.copy()
    huge[0, 3] = 1e300
    with pytest.raises(v.VoteError):
        s.solve(torch.from_numpy(huge).cuda())
    r = s.solve(dev(p))
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    assert r["depth"] == o["depth"]


def test_injected_allocation_failure_is_reported_and_recoverable():
    v = vote_mod()
    p = small(inputs.POSE3DOF, 500, 11)
    s = v.Solver(p.family, p.eps, p.bounds)
    s.set_option(v.VOTE_OPT_FAULT_ALLOC_AT, 3)
    with pytest.raises(v.VoteError) as ei:
        s.solve(dev(p))
    assert ei.value.code == 2
    s.set_option(v.VOTE_OPT_FAULT_ALLOC_AT, 0)
    r = s.solve(dev(p))
    assert r["depth"] == oracle.solve(p.family, p.eps, p.bounds, p.params)["depth"]


def test_solve_host_equals_solve_device():
    v = vote_mod()
    p = small(inputs.PLANE3D_SPH, 800, 12)
    s = v.Solver(p.family, p.eps, p.bounds)
    a = s.solve(dev(p))
    b = s.solve_host(p.params)
    assert a["depth"] == b["depth"]
    assert np.array_equal(a["best_leaf"], b["best_leaf"])
    assert np.array_equal(v.mask_words_to_numpy(a["mask"]), b["mask"])
