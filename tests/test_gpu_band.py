"""Screen band, bounded waits and grouping statistics of the CUDA path, through the C ABI.

* Screen band: inputs on a coarse dyadic grid (with repeats) put residuals exactly
  on the UB and LB radii and exactly on snap-bin edges (rounding ties), i.e. inside
  the FP32 screen's error band (Sec. 3.2's test, with the canonization's rounding).
  The FP64 recheck must run (rechecks > 0) and both precision modes must equal the
  oracle bit for bit.
* Bounded waits: with the spin limit at 0 every proximity kernel gives up on its
  first bulk copy; the solve returns VOTE_ETIMEOUT and the context then solves
  normally again.
* Grouping statistics: records entering the grouping (the canonization's merge of
  equal canonical surfaces) and canonical records leaving it, per level.
"""
import numpy as np
import pytest

import oracle
from paper_2107_11810_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FAMS = [inputs.LINE2D, inputs.PLANE3D_SPH, inputs.POSE3DOF, inputs.RAYS3D, inputs.POINTSET2D, inputs.AFFINE4D]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11810_gb300 import build
    build.build()


def vote_mod():
    from paper_2107_11810_gb300 import vote
    return vote


def dyadic_problem(family, seed):
    """A small problem of the family whose parameters are rounded to a coarse dyadic
    grid: many exact ties between residuals, radii and snap-bin edges."""
    if family == inputs.LINE2D:
        p = inputs.line2d(n=3000, inlier_frac=0.3, eps=2.0 ** -6, quantize=6, seed=seed)
        return p, p.params
    if family == inputs.PLANE3D_SPH:
        p = inputs.plane3d(n=2500, inlier_frac=0.3, eps=0.0625, sigma=0.002, seed=seed)
        return p, np.round(p.params * 16.0) / 16.0
    if family == inputs.RAYS3D:
        p = inputs.rays3d(n=3000, inlier_frac=0.3, eps=2.0 ** -6, noise=0.002, seed=seed)
        return p, np.round(p.params * 64.0) / 64.0
    if family == inputs.POINTSET2D:
        p = inputs.pointset2d(m=50, eps=2.0 ** -5, noise=0.002, seed=seed)
        return p, np.round(p.params * 64.0) / 64.0
    if family == inputs.AFFINE4D:
        p = inputs.affine4d(n=1500, inlier_frac=0.3, eps=2.0 ** -3, noise=0.005, seed=seed)
        return p, np.round(p.params * 64.0) / 64.0
    p = inputs.pose3dof(n=3000, inlier_frac=0.3, eps_xy=1.0, eps_yaw_deg=2.0, noise_deg=0.05, seed=seed)
    q = p.params.copy()
    q[:2] = np.round(q[:2] * 4.0) / 4.0          # w1, w2 (m)
    q[2:] = np.round(q[2:] * 8.0) / 8.0          # a, b (m)
    return p, q


def solve(v, p, params, precision, **opts):
    s = v.Solver(p.family, p.eps, p.bounds, precision=precision)
    for k, val in opts.items():
        s.set_option(getattr(v, k), val)
    r = s.solve(torch.from_numpy(np.ascontiguousarray(params)).cuda())
    r["mask"] = v.mask_words_to_numpy(r["mask"])
    return r, s


def assert_same(g, o, n):
    assert g["depth"] == o["depth"]
    assert np.array_equal(g["best_leaf"], o["best_leaf"])
    assert np.array_equal(g["best_point"], o["best_point"])
    assert np.array_equal(g["mask"][: (n + 31) // 32], o["mask"])


@pytest.mark.parametrize("family", FAMS)
def test_screen_band_rechecks_and_parity(family):
    v = vote_mod()
    p, params = dyadic_problem(family, 2107 + family)
    o = oracle.solve(p.family, p.eps, p.bounds, params)
    r1, s1 = solve(v, p, params, 1)
    r0, s0 = solve(v, p, params, 0)
    assert_same(r1, o, params.shape[1])
    assert_same(r0, o, params.shape[1])
    assert s1.stats()["rechecks"] > 0            # the band was entered and rechecked
    assert s0.stats()["rechecks"] == 0           # plain FP64 has no screen
    assert s1.stats()["tests"] == s0.stats()["tests"]


@pytest.mark.parametrize("precision", [0, 1])
def test_spin_limit_gives_timeout_and_context_recovers(precision):
    v = vote_mod()
    p = inputs.plane3d(n=3000, inlier_frac=0.2, eps=0.06, sigma=0.002, seed=77)
    o = oracle.solve(p.family, p.eps, p.bounds, p.params)
    s = v.Solver(p.family, p.eps, p.bounds, precision=precision)
    t = torch.from_numpy(np.ascontiguousarray(p.params)).cuda()
    s.set_option(v.VOTE_OPT_SPIN_LIMIT, 0)
    with pytest.raises(v.VoteError) as e:
        s.solve(t)
    assert e.value.code == 5                     # VOTE_ETIMEOUT
    torch.cuda.synchronize()                     # the context is still usable
    s.set_option(v.VOTE_OPT_SPIN_LIMIT, 1 << 22)
    r = s.solve(t)
    r["mask"] = v.mask_words_to_numpy(r["mask"])
    assert_same(r, o, p.n)
    with pytest.raises(v.VoteError):
        s.set_option(v.VOTE_OPT_SPIN_LIMIT, -1)


def test_grouping_level_statistics():
    v = vote_mod()
    p = inputs.plane3d(n=2500, inlier_frac=0.2, eps=0.06, sigma=0.002, seed=15)
    params = np.concatenate([p.params, p.params[:, :700], p.params[:, :300]], axis=1)
    n = params.shape[1]
    o = oracle.solve(p.family, p.eps, p.bounds, params)
    r, s = solve(v, p, params, 1, VOTE_OPT_GROUP=1)
    assert_same(r, o, n)
    ls = s.level_stats()
    gin, gout = ls["grouped_in"], ls["grouped_out"]
    assert gin[0] == n                           # every lifted record enters the root's grouping
    assert gout[0] <= 2500                       # the 1000 repeats merge with their originals
    assert np.all(gout <= gin) and np.all(gout >= 0)
    r0, s0 = solve(v, p, params, 1)
    ls0 = s0.level_stats()
    assert not ls0["grouped_in"].any() and not ls0["grouped_out"].any()
    assert np.array_equal(ls0["cells"] > 0, ls0["records"] > 0)
