"""Write complete oracle solves of configuration-size problems to tests/golden/.

* plane3d_eps005_n1e4: the plane workload's configuration (eps_d = 0.005, so
  L = 12 levels) at 1e4 points;
* pose6dof_n5000: the calibrated-camera configuration (5,000 matches, 250
  inliers, +-30 deg rotation prior, 10 m translation box, 7 levels, constant
  vertical tolerance), and pose6dof_prior5_n5000, the same with a +-5 deg prior;
* radial5dof_n5000: the radial camera (Sec. 4.2.4) at the same sizes;
* pointset2d_m300, affine4d_n1e4: the point-set (300 x 300 points) and affine
  4-space (1e4 points) benchmark workloads.

Each is Algorithm 2 with canonization (Sec. 3.2) and pruning (Sec. 3.3), solved by
the multi-core oracle (OpenMP over root subtrees; its results equal the
single-thread oracle's, which the CPU suite checks).  A solve takes minutes on a
workstation, too long to repeat in every GPU test run, so the result is stored
together with the SHA-256 of the generated input: the GPU test compares with the
stored result when its regenerated input has the same hash, and runs the oracle
itself otherwise.

    python tests/golden/make_full_eps.py [case ...]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2107_11810_gb300 import inputs  # noqa: E402

CASES = {
    # eps 0.005 and the seed are the plane workload's defaults
    "plane3d_eps005_n1e4": dict(generator="plane3d", kwargs=dict(n=10_000, inlier_frac=0.05)),
    "pose6dof_prior5_n5000": dict(generator="pose6dof", kwargs=dict(n=5000, prior_deg=5.0)),
    "pose6dof_n5000": dict(generator="pose6dof", kwargs=dict(n=5000, prior_deg=30.0)),
    "radial5dof_n5000": dict(generator="radial5dof", kwargs=dict(n=5000)),
    "pointset2d_m300": dict(generator="pointset2d", kwargs=dict(m=300)),
    "affine4d_n1e4": dict(generator="affine4d", kwargs=dict()),
}
for _c in CASES.values():
    _c["make"] = (lambda c: lambda: getattr(inputs, c["generator"])(**c["kwargs"]))(_c)
NAME = "plane3d_eps005_n1e4"
KWARGS = CASES[NAME]["kwargs"]


def params_sha256(params: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(params, dtype="<f8").tobytes()).hexdigest()


def write(name):
    case = CASES[name]
    p = case["make"]()
    t0 = time.perf_counter()
    r = oracle.solve_parallel(p.family, p.eps, p.bounds, p.params)
    dt = time.perf_counter() - t0
    st = r["stats"]
    out = dict(name=name, generator=case["generator"], kwargs=case["kwargs"], family=p.family, n=p.n,
               params_sha256=params_sha256(p.params),
               source="oracle/gv_oracle.c, multi-core solve (Algorithm 2, Sec. 3.2 canonization, Sec. 3.3 "
                      "pruning)",
               depth=r["depth"], best_leaf=[int(x) for x in r["best_leaf"]],
               best_point=[float(x).hex() for x in r["best_point"]],
               mask=[int(x) for x in r["mask"]],
               oracle_tests=int(st[0]), oracle_threads=int(st[4]), oracle_seconds=round(dt, 1))
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(f"{path}: depth {r['depth']}, {int(st[0])} tests, {dt:.1f} s on {int(st[4])} threads")


def main():
    for name in sys.argv[1:] or sorted(CASES):
        write(name)


if __name__ == "__main__":
    main()
