"""One solve of a seeded synthetic workload, as a small target for profiler captures.

    python -m paper_2107_11810_gb300.profile_case --family plane3d --n 100000 --chunk 6000000

builds the library if needed, runs one ``Solver.solve`` on ``cuda:0`` and prints one
JSON line (depth, wall time, chunks, kernel launches, tests).  The inputs are the
generators of :mod:`paper_2107_11810_gb300.inputs` with their default parameters and
``n`` points.
"""
from __future__ import annotations

import argparse
import json
import time

from . import build, inputs

GENERATORS = {
    "plane3d": lambda n, seed: inputs.plane3d(n=n, seed=seed),
    "pose3dof": lambda n, seed: inputs.pose3dof(n=n, seed=seed),
    "line2d": lambda n, seed: inputs.line2d(n=n, seed=seed),
}


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--family", choices=sorted(GENERATORS), default="plane3d")
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--chunk", type=int, default=0, help="records per chunk (0: library default)")
    ap.add_argument("--seed", type=int, default=inputs.SEED_BASE + 1)
    ap.add_argument("--precision", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    from . import vote
    build.build()
    p = GENERATORS[args.family](args.n, args.seed)
    kw = dict(precision=args.precision)
    if args.chunk > 0:
        kw["chunk_records"] = args.chunk
    s = vote.Solver(p.family, p.eps, p.bounds, **kw)
    t = torch.from_numpy(p.params).cuda()
    torch.cuda.synchronize()
    t0 = time.time()
    r = s.solve(t)
    torch.cuda.synchronize()
    st = s.stats()
    out = dict(family=args.family, n=args.n, chunk=args.chunk, depth=r["depth"], sec=time.time() - t0,
               chunks=st["chunks"], launches=st["launches"], tests=st["tests"])
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
