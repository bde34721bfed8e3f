"""The engine's level structure (its own host code, written separately from the
oracle) equals the oracle's, on the CPU through vote_level_constants: levels and
splits per coordinate, the snap steps of the dependent residuals and of the
essential parameters, and the accumulated canonization error bound (Sec. 3.2,
"Canonization" and the eps update).  The GPU parity tests rely on these being
identical bit for bit; this checks it for every family without a device, on the
benchmark workloads and on small instances with few levels.
"""
import numpy as np
import pytest

import oracle
from paper_2107_11810_gb300 import inputs

CASES = {
    "line2d": lambda: inputs.line2d(n=10),
    "plane3d": lambda: inputs.plane3d(n=10),
    "plane3d_coarse": lambda: inputs.plane3d(n=10, eps=0.08),
    "pose3dof": lambda: inputs.pose3dof(n=10),
    "pose6dof": lambda: inputs.pose6dof(n=10),
    "pose6dof_3levels": lambda: inputs.pose6dof(n=10, levels=3),
    "rays3d": lambda: inputs.rays3d(n=10),
    "pointset2d": lambda: inputs.pointset2d(m=4),
    "affine4d": lambda: inputs.affine4d(n=10),
    "radial5dof": lambda: inputs.radial5dof(n=10),
    "radial5dof_3levels": lambda: inputs.radial5dof(n=10, levels=3),
}


@pytest.fixture(scope="module")
def vote():
    from paper_2107_11810_gb300 import build, vote as v
    build.build()
    return v


@pytest.mark.parametrize("name", sorted(CASES))
def test_engine_level_constants_equal_the_oracle(vote, name):
    p = CASES[name]()
    e = vote.level_constants(p.family, p.eps, p.bounds)
    o = oracle.levels(p.family, p.eps, p.bounds)
    L = o["L"]
    assert e["L"] == L
    assert np.array_equal(e["Lj"], o["Lj"])
    assert np.array_equal(e["s_f"], o["s_f"])
    assert np.array_equal(e["s_t"], o["s_t"][:L])
    assert np.array_equal(e["A"], o["A"][1:L + 1])


def test_level_constants_reject_bad_input(vote):
    with pytest.raises(vote.VoteError):
        vote.level_constants(inputs.LINE2D, [0.0, 0.01], [-1.0, 1.0, -1.0, 2.0])
    with pytest.raises(vote.VoteError):
        vote.level_constants(inputs.LINE2D, [0.01, 0.01], [1.0, -1.0, -1.0, 2.0])
