"""Soft inlier score on the GPU against the plain-PyTorch FP64 oracle, autograd
checks, and refinement inside the best leaf."""
import numpy as np
import pytest

from oracle import softscore as oss
from paper_2107_11810_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_11810_gb300 import build
    build.build()


CASES = [
    (inputs.LINE2D, lambda: inputs.line2d(n=3001, seed=41), [0.02]),
    (inputs.PLANE3D_SPH, lambda: inputs.plane3d(n=5003, seed=42), [0.01]),
    (inputs.POSE3DOF, lambda: inputs.pose3dof(n=4007, seed=43), [0.5, 0.5]),
    (inputs.POSE6DOF, lambda: inputs.pose6dof(n=1503, prior_deg=5.0, levels=5, seed=44), [0.1, 0.1]),
    (inputs.RAYS3D, lambda: inputs.rays3d(n=4001, seed=45), [0.01, 0.01]),
    (inputs.POINTSET2D, lambda: inputs.pointset2d(m=60, eps=0.02, seed=46), [0.02, 0.02]),
    (inputs.AFFINE4D, lambda: inputs.affine4d(n=3001, eps=0.1, seed=47), [0.05]),
]


def setup(fam, mk, tol, masked):
    from paper_2107_11810_gb300 import vote
    p = mk()
    s = vote.Solver(p.family, p.eps, p.bounds)
    prm = torch.from_numpy(p.params).cuda()
    rng = np.random.default_rng(fam)
    w = rng.integers(0, 2, p.n).astype(np.float64) if masked else np.ones(p.n)
    bits = np.packbits(w.astype(np.uint8), bitorder="little")
    bits = np.concatenate([bits, np.zeros((-len(bits)) % 4, np.uint8)])
    mask = torch.from_numpy(bits.view(np.int32).copy()).cuda() if masked else None
    pt = torch.tensor(p.truth + 0.37 * np.array(tol[:1] * p.d), dtype=torch.float64)
    return p, s, prm, w, mask, pt


@pytest.mark.parametrize("fam,mk,tol", CASES)
@pytest.mark.parametrize("masked", [False, True])
def test_forward_backward_match_oracle(fam, mk, tol, masked):
    from paper_2107_11810_gb300.softscore import SoftScore
    p, s, prm, w, mask, pt = setup(fam, mk, tol, masked)
    ptg = pt.cuda().requires_grad_(True)
    prmg = prm.clone().requires_grad_(True)
    out = SoftScore.apply(ptg, prmg, s, mask, tol)
    out.backward()
    po = pt.clone().requires_grad_(True)
    qo = torch.from_numpy(p.params.copy()).requires_grad_(True)
    ref = oss.softscore(fam, qo, po, torch.from_numpy(w), tol)
    ref.backward()
    o, r = float(out.detach()), float(ref.detach())
    assert abs(o - r) <= 1e-12 * max(1.0, abs(r))
    assert torch.allclose(ptg.grad.cpu(), po.grad, rtol=1e-10, atol=1e-10)
    assert torch.allclose(prmg.grad.cpu(), qo.grad, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("fam,mk,tol", CASES)
def test_gradcheck_and_central_differences(fam, mk, tol):
    from paper_2107_11810_gb300.softscore import SoftScore
    p, s, prm, w, mask, pt = setup(fam, mk, tol, False)
    small = prm[:, :64].contiguous().clone().requires_grad_(True)
    ptg = pt.cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: SoftScore.apply(a, b, s, None, tol), (ptg, small),
                                    eps=1e-6, atol=1e-6, rtol=1e-5)
    # central differences of the GPU forward, h = 1e-6
    g = torch.autograd.grad(SoftScore.apply(ptg, prm, s, None, tol), ptg)[0].cpu()
    h = 1e-6
    for j in range(p.d):
        e = torch.zeros(p.d, dtype=torch.float64, device="cuda")
        e[j] = h
        fd = (SoftScore.apply(ptg.detach() + e, prm, s, None, tol) -
              SoftScore.apply(ptg.detach() - e, prm, s, None, tol)) / (2 * h)
        assert abs(float(fd) - float(g[j])) <= 1e-5 * max(1.0, abs(float(fd)))


@pytest.mark.parametrize("fam,mk,tol", CASES)
def test_refine_improves_score_inside_the_best_leaf(fam, mk, tol):
    from paper_2107_11810_gb300.softscore import SoftScore
    p, s, prm, w, mask, pt = setup(fam, mk, tol, False)
    r = s.solve(prm)
    lo, hi = s.leaf_box(r["best_leaf"])
    assert np.all(r["best_point"] >= lo) and np.all(r["best_point"] <= hi)
    start = SoftScore.apply(torch.from_numpy(r["best_point"]).cuda(), prm, s, r["mask"], None)
    q, score = s.refine(prm, r["mask"], lo, hi, r["best_point"], iters=50)
    assert np.all(q >= lo) and np.all(q <= hi)
    assert score >= float(start) - 1e-12
    again = SoftScore.apply(torch.from_numpy(q).cuda(), prm, s, r["mask"], None)
    assert abs(float(again) - score) <= 1e-12 * max(1.0, score)
