"""Write the golden fixtures of tests/golden/ from the oracle only.

The paper prints no worked example (its figures are lost and its tables are CPU
runtimes on unavailable datasets), so these fixtures are regression values of the
oracle (plain FP64 C implementation of Algorithm 2 with canonization, Sec. 3.2,
and pruning, Sec. 3.3) on small seeded instances of each family.  They let the CPU
and GPU suites detect any change of results without rerunning the oracle.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2107_11810_gb300 import inputs  # noqa: E402

CASES = [
    ("line2d_n500", "line2d", dict(n=500, inlier_frac=0.2, eps=0.01, seed=101)),
    ("plane3d_n400", "plane3d", dict(n=400, inlier_frac=0.2, eps=0.04, sigma=0.002, seed=102)),
    ("pose3dof_n600", "pose3dof", dict(n=600, inlier_frac=0.2, eps_xy=0.5, eps_yaw_deg=1.0, seed=103)),
]


def main():
    for name, gen, kw in CASES:
        p = getattr(inputs, gen)(**kw)
        r = oracle.solve(p.family, p.eps, p.bounds, p.params)
        # the input arrays are stored too (hex floats), so the fixture does not depend
        # on the platform's libm used by the generators
        out = dict(name=name, generator=gen, kwargs=kw, family=p.family, n=p.n,
                   eps=[float(x).hex() for x in p.eps], bounds=[float(x).hex() for x in p.bounds],
                   params=[[float(x).hex() for x in row] for row in p.params],
                   source="oracle/gv_oracle.c (Algorithm 2, Sec. 3.2 canonization, Sec. 3.3 pruning); "
                          "the paper prints no worked example",
                   depth=r["depth"], best_leaf=[int(x) for x in r["best_leaf"]],
                   best_point=[float(x).hex() for x in r["best_point"]],
                   mask=[int(w) for w in r["mask"]])
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=0)
        print(name, r["depth"], r["best_leaf"].tolist())


if __name__ == "__main__":
    main()
