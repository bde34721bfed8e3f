"""Pin of the oracle on 2D lines by exact rational arithmetic.

For lines every step of the recursion works on dyadic numbers of short mantissa:
the snap steps are powers of two, the child shift in m is a power of two (the m
range has width 2), the shift in b has a two-bit mantissa (width 3), so snapping
and the child residual f' = (f~ - t~ dm) - db are exact in FP64.  Here the whole
recursion of Algorithm 2 with canonization (Sec. 3.2: snap f to s_f and t to
s_t(l), merge equal snapped surfaces, test each child against "eps plus the cell
radius" plus the accumulated canonization error A_{l+1}) is restated with
Python's Fraction, and every cell's UB/LB count without pruning must equal the
oracle's, as must the best leaf and its depth.  The level constants (h, s_f, s_t,
A) and the FP64 lift at the root are inputs of the definition; they are taken from
the oracle and pinned separately (level structure, brute-force depth).  The radii
(eps + h' + |t~| h'_m + A and eps - A) are formed exactly here, while the oracle
rounds them in FP64, so the comparison also shows that this rounding never
changes a decision on these inputs.
"""
import dataclasses
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2107_11810_gb300 import inputs


def exact_search(p):
    lv = oracle.levels(p.family, p.eps, p.bounds)
    L, Lj = lv["L"], [int(x) for x in lv["Lj"]]
    h = [[Fr(float(x)) for x in row] for row in lv["h"]]
    s_f = Fr(float(lv["s_f"][0]))
    s_t = [Fr(float(x)) for x in lv["s_t"][:, 0]]
    A = [Fr(float(x)) for x in lv["A"][:, 0]]
    eps_b = Fr(float(p.eps[1]))
    f0, t0 = oracle.root_records(p.family, p.eps, p.bounds, p.params)
    recs = [(Fr(float(f0[0, i])), Fr(float(t0[0, i])), 1) for i in range(p.n)]
    trace = {}
    best = {"ub": 0, "leaf": None}

    def visit(l, ci, recs):
        if l == L:
            ub = sum(m for _, _, m in recs)
            if ub and (ub > best["ub"] or (ub == best["ub"] and tuple(ci) < best["leaf"])):
                best["ub"], best["leaf"] = ub, tuple(ci)
            return
        merged = {}
        for f, t, m in recs:                       # canonize: snap (round half to even), merge
            key = (round(f / s_f), round(t / s_t[l]))
            merged[key] = merged.get(key, 0) + m
        canon = [(qf * s_f, qt * s_t[l], m) for (qf, qt), m in merged.items()]
        for b in range(4):
            if any(((b >> j) & 1) and l >= Lj[j] for j in range(2)):
                continue
            cc, sh = [], []
            for j in range(2):
                if l < Lj[j]:
                    bit = (b >> j) & 1
                    cc.append(2 * ci[j] + bit)
                    sh.append(h[l + 1][j] if bit else -h[l + 1][j])
                else:
                    cc.append(ci[j])
                    sh.append(Fr(0))
            ub = lb = 0
            kids = []
            for f, t, m in canon:
                fo = (f - t * sh[0]) - sh[1]
                a = abs(fo)
                if a <= eps_b + h[l + 1][1] + abs(t) * h[l + 1][0] + A[l + 1]:
                    ub += m
                    kids.append((fo, t, m))
                if a <= eps_b - A[l + 1]:
                    lb += m
            trace[(l + 1, tuple(cc))] = (ub, lb)
            if ub:
                visit(l + 1, cc, kids)

    visit(0, [0, 0], recs)
    return trace, best


@pytest.mark.parametrize("n,seed,eps", [(40, 31, 0.01), (50, 32, 0.02), (30, 33, 0.01)])
def test_line_counts_equal_exact_rational_recursion(n, seed, eps):
    p = inputs.line2d(n=n, inlier_frac=0.3, eps=eps, seed=seed)
    trace, best = exact_search(p)
    o = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=oracle.NO_PRUNE, trace_cap=2_000_000)
    to = o["trace"]
    got = {(int(l), tuple(int(x) for x in c)): (int(u), int(b))
           for l, c, u, b in zip(to["level"], to["coords"], to["ub"], to["lb"])}
    assert len(got) == len(to["level"]) > 100
    assert got == trace
    assert o["depth"] == best["ub"]
    assert tuple(int(x) for x in o["best_leaf"]) == best["leaf"]


def test_exact_recursion_sees_merges():
    # duplicated surfaces must merge into one canonical record with summed multiplicity
    p = inputs.line2d(n=20, inlier_frac=0.5, eps=0.02, seed=34)
    dup = np.concatenate([p.params, p.params[:, :7]], axis=1)
    q = dataclasses.replace(p, params=dup)
    trace, best = exact_search(q)
    o = oracle.solve(q.family, q.eps, q.bounds, q.params, flags=oracle.NO_PRUNE, trace_cap=2_000_000)
    to = o["trace"]
    got = {(int(l), tuple(int(x) for x in c)): (int(u), int(b))
           for l, c, u, b in zip(to["level"], to["coords"], to["ub"], to["lb"])}
    assert got == trace
    assert o["depth"] == best["ub"] >= 14          # the 7 duplicated surfaces count twice


# Planted mistakes that only move a margin or a tie: the brute-force pins can miss
# them (they change results only near a decision), the exact per-cell comparison
# must not.  The level constants and root records still come from the unmodified
# oracle, so only the recursion is under test.
EXACT_MUTANTS = {
    "ub_radius_without_A": ("R = R + p->A[l + 1][j];", "R = R + 0.0 * p->A[l + 1][j];"),
    "lb_radius_without_A": ("double rl = p->eps[jj] - p->A[l + 1][j];", "double rl = p->eps[jj];"),
    "snap_t_half_away": ("double q = rint(r->t[m] / p->s_t[l][m]);", "double q = round(r->t[m] / p->s_t[l][m]);"),
    "merge_keeps_one_mult": ("for (int64_t x = a; x < b; ++x) mult += recs[idx[x]].mult;",
                             "mult = recs[idx[a]].mult;"),
}


def _oracle_trace(p, lib):
    o = oracle.solve(p.family, p.eps, p.bounds, p.params, flags=oracle.NO_PRUNE, trace_cap=2_000_000, lib=lib)
    to = o["trace"]
    return {(int(l), tuple(int(x) for x in c)): (int(u), int(b))
            for l, c, u, b in zip(to["level"], to["coords"], to["ub"], to["lb"])}


@pytest.mark.parametrize("name", sorted(EXACT_MUTANTS))
def test_exact_pin_catches_margin_and_tie_mistakes(name):
    old, new = EXACT_MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    lib = oracle.load_variant(src.replace(old, new), "exact_" + name)
    caught = False
    for n, seed in ((40, 31), (50, 32)):
        p = inputs.line2d(n=n, inlier_frac=0.3, eps=0.02, seed=seed)
        if name == "merge_keeps_one_mult":
            p = dataclasses.replace(p, params=np.concatenate([p.params, p.params[:, :9]], axis=1))
        trace, _ = exact_search(p)
        if _oracle_trace(p, lib) != trace:
            caught = True
            break
    assert caught, f"mutant {name} survived the exact pin"
