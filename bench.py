"""Benchmark of the voting hot path on GB300.

One step = one complete solve (lift, every level's snap / proximity test /
prune / split, leaf argmax, inlier-mask replay) of one synthetic problem shaped
like the paper's workloads; the default is 3D plane fitting with 1,000,000
points (2 % on a plane, eps = 0.005, (theta, phi, d) space).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl gv|reference] [--no-fp64] [--no-cpu] [--no-group-stats]

After the timed steps, one plain-FP64 solve of the same workload checks that the
two precision modes give identical results and times it (the metric's
comparison), one solve with grouping on reports the grouping's merge fraction per
level, and the oracle (plain FP64 C on the host cores) is timed on a bounded
sample.  Prints one JSON line (rank 0).  Under torchrun every rank solves its own copy
of the problem (independent problems, no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2107_11810_gb300 import inputs  # noqa: E402

METRIC = "solved problems/sec and surface-cell tests/sec: FP32+recheck vs plain FP64 path"

WORKLOADS = {
    "plane3d_n1e6": dict(make=lambda: inputs.plane3d(), desc="3D plane fitting, 1e6 points in the unit cube, "
                         "2% inliers (sigma 0.001), eps_d=0.005, eps_angle=eps/sqrt3, (theta,phi,d) space",
                         group_sample=lambda: inputs.plane3d(n=10_000)),
    "pose3dof_n1e6": dict(make=lambda: inputs.pose3dof(), desc="3DoF camera voting, 1e6 matches, 1% inliers, "
                          "eps 0.25 m / 0.5 deg, (yaw,x,y) space", group_sample=lambda: inputs.pose3dof(n=100_000)),
    "line2d_n1e4": dict(make=lambda: inputs.line2d(), desc="2D line fitting, 1e4 points, 10% inliers, eps 0.01, "
                        "(m,b) space"),
    "plane3d_n1e4": dict(make=lambda: inputs.plane3d(n=10_000), desc="3D plane fitting, 1e4 points (the plane "
                         "workload's shape at a hundredth of its size; a whole solve is a small profiler capture)"),
    "plane3d_n1e5": dict(make=lambda: inputs.plane3d(n=100_000), desc="3D plane fitting, 1e5 points (the plane "
                         "workload's shape at a tenth of its size; a small target for profiler captures)"),
    "pose3dof_n3e5": dict(make=lambda: inputs.pose3dof(n=300_000), desc="3DoF camera voting, 3e5 matches (a small "
                          "target for profiler captures)"),
    "pose6dof_n5000": dict(make=lambda: inputs.pose6dof(n=5000, prior_deg=30.0), desc="6DoF calibrated-camera "
                           "voting, 5,000 matches (250 inliers, 0.1 deg bearing noise), rotation prior +-30 deg per "
                           "axis, 10 m translation box, 7 levels per coordinate, constant vertical tolerance "
                           "box/128 in x and y, (phi1,phi2,phi3,z,x,y) space"),
    "pose6dof_prior5_n5000": dict(make=lambda: inputs.pose6dof(n=5000, prior_deg=5.0), desc="6DoF calibrated-"
                                  "camera voting as pose6dof_n5000 with a +-5 deg rotation prior"),
    "rays3d_n1e5": dict(make=lambda: inputs.rays3d(), desc="rays in 3-space, 1e5 rays (2% through a common "
                        "point, N(0, 0.0005) offsets), slopes U[-2,2], unit cube, eps 0.002, (x,y,z) space"),
    "pointset2d_m300": dict(make=lambda: inputs.pointset2d(m=300), desc="point-set similarity alignment, two sets of "
                            "300 points (B = s R A + t + N(0, 0.002)), all 90,000 pairs as surfaces, eps 0.01, "
                            "(c,d,a,b) space"),
    "affine4d_n1e4": dict(make=lambda: inputs.affine4d(), desc="hyperplane fitting in 4-space (affine form), 1e4 "
                          "points, 5% on a hyperplane (N(0, 0.002) in x4), eps 0.02, (a1,a2,a3,b) space"),
    "pose3dof_batch256": dict(make=lambda: inputs.pose3dof_batch(), batched=True,
                              desc="256 independent 3DoF problems, n log-uniform in [1e3, 1e6], inlier ratio "
                                   "U[0.5%, 5%]; one vote_solve_batched call per step"),
}
# FP32-pipe instructions per (child cell, canonical surface) test, counted from
# the formulas of each family's residual and comparisons
INSTR_PER_TEST = {inputs.LINE2D: 7, inputs.PLANE3D_SPH: 10, inputs.POSE3DOF: 14, inputs.POSE6DOF: 30,
                  inputs.RAYS3D: 10, inputs.POINTSET2D: 10, inputs.AFFINE4D: 10}


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return dict(hbm_gbs=float(m["hbm_gbs"]), sm_max_mhz=float(m.get("sm_max_mhz", 2070.0)), src="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unsampled"], samples=0)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(self.samples))


KERNEL_SOURCES = {"k_count": ("gv_count.cu", "gv_tile.cuh", "gv_device.cuh", "gv_kernels.h"),
                  "k_emit": ("gv_emit.cu", "gv_tile.cuh", "gv_device.cuh", "gv_kernels.h")}


def kernel_hash(kernel: str):
    """sha256 (first 16 hex digits) of the sources a kernel is built from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2107_11810_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, family: str, algorithmic_bytes_per_launch: float):
    """DRAM traffic per launch of a kernel: the ratio of ncu's dram bytes (read + write)
    to the launch's algorithmic bytes, measured on a smaller case of the same kernel
    and committed in profiles/ncu_traffic.txt, times this run's algorithmic bytes per
    launch.  None once the kernel sources differ from the ones captured."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    kh = kernel_hash(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kh and parts[1] == kernel \
                and parts[2] == family:
            return float(parts[3]) * algorithmic_bytes_per_launch
    return None


def oracle_sample(p, budget_s: float):
    """The oracle (plain FP64 C) on a bounded sample of the workload: the first n_s
    surfaces, n_s grown until one single-thread solve takes about budget_s/4
    seconds; then the same sample on every host core (OpenMP over subtrees).
    Returns dict(single=(tests/s, s), multi=(tests/s, s, threads), n_s, tests)."""
    import oracle
    n_s = 200
    while True:
        sub = np.ascontiguousarray(p.params[:, :n_s])
        t0 = time.perf_counter()
        r = oracle.solve(p.family, p.eps, p.bounds, sub)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or n_s >= p.n:
            break
        n_s = min(p.n, int(n_s * max(1.5, min(8.0, (budget_s / 4) / max(dt, 1e-3)))))
    tests = int(r["stats"][0])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    rp = oracle.solve_parallel(p.family, p.eps, p.bounds, sub, threads=cores)
    dtp = time.perf_counter() - t0
    assert rp["depth"] == r["depth"]
    # the parallel run prunes differently; its rate is taken on the serial test count
    return dict(single=(tests / dt, dt), multi=(tests / dtp, dtp, int(rp["stats"][4])), n_s=n_s, tests=tests)


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, on the host cores."""
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    p = w["make"]()
    import oracle
    oracle.build()
    smp = oracle_sample(p, 8.0)
    n_s, tests = smp["n_s"], smp["tests"]
    cores = os.cpu_count() or 1
    gpu_tests = args.ref_tests_per_problem
    sub = np.ascontiguousarray(p.params[:, :n_s])
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle.solve_parallel(p.family, p.eps, p.bounds, sub, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve_parallel(p.family, p.eps, p.bounds, sub, threads=cores)
        times.append(time.perf_counter() - t0)
    tps = tests / statistics.mean(times)
    # scale: problems/s = oracle tests/s / tests one full-size problem needs
    value = tps / gpu_tests if gpu_tests else None
    line = dict(metric=METRIC,
                value=value, unit="problems/s", impl="reference", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000 * statistics.mean(times), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, desc=w["desc"]),
                tests_per_s=tps,
                cpu_baseline=dict(value=value, unit="problems/s", cores=cores, kind="oracle",
                                  sample=f"oracle (OpenMP over subtrees, {cores} threads) solving the first {n_s} "
                                         f"of {p.n} surfaces ({tests} tests); problems/s = oracle tests/s / "
                                         f"{gpu_tests} tests per full problem",
                                  single_thread=dict(value=smp["single"][0] / gpu_tests if gpu_tests else None,
                                                     tests_per_s=smp["single"][0], cores=1)),
                e2e=dict(value=value, unit="problems/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, w):
    """Batched workload: every rank solves its greedy share of the problems with one
    vote_solve_batched call per step (no collective on the data path)."""
    import torch
    from paper_2107_11810_gb300 import shard, vote
    probs = w["make"]()
    mine = shard.partition([p.n for p in probs], world)[rank]
    local = [probs[i] for i in mine]
    p0 = probs[0]
    s = vote.Solver(p0.family, p0.eps, p0.bounds, precision=args.precision,
                    stream=torch.cuda.current_stream())
    flat, offs = vote.pack_batch([p.params for p in local])
    data = torch.from_numpy(flat).cuda()
    for _ in range(args.warmup):
        res = s.solve_batched((data, offs))
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    times, lats, launches = [], [], 0
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = s.solve_batched((data, offs))
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            lats.extend(res["latency_ms"].tolist())
            launches += int(s.stats()["launches"])
    total = sum(times)
    if world > 1:
        t = torch.tensor([total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    pinned = torch.from_numpy(flat).pin_memory()
    t0 = time.perf_counter()
    r2 = s.solve_batched((pinned.cuda(non_blocking=True), offs))
    words = torch.empty(r2["masks"].numel(), dtype=torch.int32).copy_(r2["masks"])
    e2e_t = time.perf_counter() - t0
    out = dict(metric=METRIC, value=len(probs) * args.steps / total,
               unit="problems/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
               ms_per_step=1000 * total / args.steps, higher_is_better=True, scaling="strong", vs_baseline=None,
               dtype="f32+f64" if args.precision == 1 else "f64", data="synthetic",
               config=dict(workload=args.workload, desc=w["desc"], problems=len(probs),
                           total_n=int(sum(p.n for p in probs)), l2="inputs and working set larger than L2"),
               latency_ms=dict(p50=float(np.percentile(lats, 50)), p99=float(np.percentile(lats, 99))),
               gpu_launches=launches, clocks=clk.summary(),
               e2e=dict(value=len(local) / e2e_t, unit="problems/s", h2d_bytes_per_step=int(flat.nbytes),
                        d2h_bytes_per_step=int(words.numel() * 4)))
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gv", choices=["gv", "reference"])
    ap.add_argument("--workload", default="plane3d_n1e6", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain-FP64 predicate solve of the same workload that follows the timed steps "
                         "(the metric's comparison: FP32 screen + FP64 recheck vs plain FP64, identical results)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-group-stats", action="store_true",
                    help="skip the grouped solve that reports the grouping's per-level merge fraction")
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--ref-tests-per-problem", type=float, default=0.0)
    args = ap.parse_args()
    rank, world, local = env_rank()
    if args.impl == "reference":
        if not args.ref_tests_per_problem:
            args.ref_tests_per_problem = REF_TESTS.get(args.workload, 0.0)
        return run_reference(args, rank, world)

    import torch
    from paper_2107_11810_gb300 import build, vote
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    w = WORKLOADS[args.workload]
    if w.get("batched"):
        run_batched(args, rank, world, w)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    p = w["make"]()
    stream = torch.cuda.current_stream()
    s = vote.Solver(p.family, p.eps, p.bounds, precision=args.precision, stream=stream,
                    chunk_records=args.chunk or None)
    s.set_option(vote.VOTE_OPT_KERNEL_TIMING, 1)
    surf = torch.from_numpy(p.params).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        r = s.solve(surf)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times, tests, kt = [], [], {}
    launches = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)                      # L2 flush between timed steps
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = s.solve(surf)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1000.0)
            st = s.stats()
            tests.append(st["tests"])
            launches += st["launches"]
            for k, v in s.kernel_times().items():
                a = kt.setdefault(k, [0.0, 0, 0.0])
                a[0] += v[0]; a[1] += v[1]; a[2] += v[2]
    total = sum(times)
    if world > 1:
        t = torch.tensor([total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    depth, leaf = r["depth"], r["best_leaf"].tolist()
    pk = peaks()
    value = world * args.steps / total
    tests_per_problem = statistics.mean(tests)
    # roofline of the dominant kernel class
    dom = max(("test_count", "test_emit"), key=lambda k: kt[k][0])
    ms, nl, by = kt[dom]
    avg_s = ms / 1000.0 / max(nl, 1)
    if dom == "test_count" and args.precision == 1:
        instr = INSTR_PER_TEST[p.family] * tests_per_problem * args.steps / max(nl, 1)
        achieved = instr / avg_s / 1e12
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        alu_peak = sms * 128 * pk["sm_max_mhz"] * 1e6 / 1e12
        roof = dict(bound="alu", achieved=achieved, peak=alu_peak, unit="TFP32-instr/s",
                    frac=achieved / alu_peak, kernel="k_count",
                    peak_src=f"{sms} SMs (device property) x 128 FP32 lanes x {pk['sm_max_mhz']:.0f} MHz max SM "
                             f"clock ({pk['src']}); thread instructions/s, no FMA doubling",
                    traffic=recorded_traffic("k_count", inputs.FAMILY_NAMES[p.family], by / max(nl, 1)),
                    bytes_per_launch=by / max(nl, 1))
    else:
        achieved = by / max(nl, 1) / avg_s / 1e9
        roof = dict(bound="hbm", achieved=achieved, peak=pk["hbm_gbs"], unit="GB/s",
                    frac=achieved / pk["hbm_gbs"], kernel="k_" + dom[5:], peak_src=pk["src"],
                    traffic=recorded_traffic("k_" + dom[5:], inputs.FAMILY_NAMES[p.family], by / max(nl, 1)),
                    bytes_per_launch=by / max(nl, 1))
    roof["share_of_step"] = kt[dom][0] / 1000.0 / total * world
    if kt["test_emit"][1]:
        e_ms, e_nl, e_by = kt["test_emit"]
        roof["emit_kernel"] = dict(kernel="k_emit", bound="hbm", achieved=e_by / (e_ms / 1000.0) / 1e9,
                                   peak=pk["hbm_gbs"], unit="GB/s",
                                   frac=e_by / (e_ms / 1000.0) / 1e9 / pk["hbm_gbs"],
                                   share_of_step=e_ms / 1000.0 / total * world,
                                   traffic=recorded_traffic("k_emit", inputs.FAMILY_NAMES[p.family],
                                                            e_by / max(e_nl, 1)))
    # end to end through the public API with host buffers
    pinned = torch.from_numpy(p.params).pin_memory()
    e2e_times = []
    for _ in range(1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rh = s.solve_host(pinned)
        e2e_times.append(time.perf_counter() - t0)
    assert rh["depth"] == depth
    e2e = dict(value=1.0 / statistics.mean(e2e_times), unit="problems/s",
               h2d_bytes_per_step=int(p.params.nbytes), d2h_bytes_per_step=int(((p.n + 31) // 32) * 4))
    out = dict(metric=METRIC, value=value, unit="problems/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
               ms_per_step=1000 * total / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
               dtype="f32+f64" if args.precision == 1 else "f64", data="synthetic",
               config=dict(workload=args.workload, desc=w["desc"], n=p.n, l2="flushed between timed steps",
                           precision="FP32 screen + FP64 recheck" if args.precision == 1 else "FP64"),
               tests_per_s=world * sum(tests) / total, tests_per_problem=tests_per_problem,
               result=dict(depth=depth, best_leaf=leaf, best_point=r["best_point"].tolist()),
               gpu_launches=launches, roofline=roof, e2e=e2e, clocks=clk.summary(),
               kernel_ms={k: round(v[0] / args.steps, 3) for k, v in kt.items() if v[1]})
    if args.no_fp64:
        out["fp64_plain"] = dict(skipped="--no-fp64")
    elif args.precision == 1:
        s.set_option(vote.VOTE_OPT_PRECISION, 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r64 = s.solve(surf)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1000.0
        same = (r64["depth"] == depth and r64["best_leaf"].tolist() == leaf and
                torch.equal(r64["mask"], r["mask"]))
        out["fp64_plain"] = dict(value=1.0 / t64, unit="problems/s", tests_per_s=s.stats()["tests"] / t64,
                                 seconds=t64, identical_results=bool(same),
                                 speedup_fp32_screen=value / world * t64,
                                 note="one plain-FP64 solve of the same workload after the timed steps")
        s.set_option(vote.VOTE_OPT_PRECISION, 1)
    if not args.no_group_stats:
        # per-level merge fraction of the canonization's grouping (records in ->
        # canonical records out): one solve with grouping on and one without, on the
        # workload's own instance when it is small, else on the same generator with
        # fewer surfaces (grouping hashes every record of every step: on the 1e6-point
        # plane that is about 1.3e12 records, hours of work)
        wg = w.get("group_sample", None)
        pg = wg() if wg else p
        sg = vote.Solver(pg.family, pg.eps, pg.bounds, precision=args.precision, stream=stream)
        tg = torch.from_numpy(pg.params).cuda()
        r0 = sg.solve(tg)
        sg.set_option(vote.VOTE_OPT_GROUP, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rg = sg.solve(tg)
        e1.record(stream)
        torch.cuda.synchronize()
        ls = sg.level_stats()
        gin, gout = ls["grouped_in"], ls["grouped_out"]
        out["grouping"] = dict(
            workload=f"{args.workload} generator at n={pg.n}" if wg else args.workload,
            seconds=e0.elapsed_time(e1) / 1000.0,
            identical_results=bool(rg["depth"] == r0["depth"] and rg["best_leaf"].tolist() == r0["best_leaf"].tolist()
                                   and torch.equal(rg["mask"], r0["mask"])),
            records_in=int(gin.sum()), records_out=int(gout.sum()),
            merge_fraction=1.0 - float(gout.sum()) / max(float(gin.sum()), 1.0),
            merge_fraction_per_level=[round(1.0 - float(o) / float(i), 6) if i else None
                                      for i, o in zip(gin.tolist(), gout.tolist())],
            note="VOTE_OPT_GROUP=1 after the timed steps; the timed path runs without grouping")
    if rank == 0 and not args.no_cpu:
        try:
            smp = oracle_sample(p, 16.0)
            tps, dtp, thr = smp["multi"]
            out["cpu_baseline"] = dict(value=tps / tests_per_problem, unit="problems/s", cores=thr, kind="oracle",
                                       tests_per_s=tps,
                                       sample=f"oracle solve of the first {smp['n_s']} of {p.n} surfaces "
                                              f"({smp['tests']} tests; {dtp:.1f} s on {thr} threads, OpenMP over "
                                              f"subtrees); problems/s = oracle tests/s / {tests_per_problem:.4g} "
                                              f"tests per full problem (GPU count)",
                                       single_thread=dict(value=smp["single"][0] / tests_per_problem,
                                                          tests_per_s=smp["single"][0], seconds=smp["single"][1],
                                                          cores=1))
        except Exception as e:   # the baseline must not sink the GPU line
            out["cpu_baseline"] = dict(value=None, unit="problems/s", cores=os.cpu_count(), kind="oracle",
                                       sample=f"failed: {e}")
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# tests per full problem measured by the GPU path (used to scale the reference
# arm's oracle sample to problems/s); refreshed from bench runs
REF_TESTS = {"plane3d_n1e6": 1.0476383009996e13, "pose3dof_n1e6": 3.0e9, "line2d_n1e4": 8.324422e6,
             "pose6dof_n5000": 6.136e11, "pose6dof_prior5_n5000": 9.504e9, "rays3d_n1e5": 1.027e8}

if __name__ == "__main__":
    main()
