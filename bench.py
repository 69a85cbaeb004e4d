"""Benchmark: Biot-Savart velocity at every node of the 64^3 Fourier workload on GB300.

One step = one velocity evaluation at all 262144 nodes over all 1500282 tets
(float32 bulk, far_ratio 2, 4-point far rule, 8 x 16 directions), i.e.
3.93e11 node-tet interactions.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): every rank evaluates its own replica of the workload
(independent problems, no collective on the data path; weak scaling); the
timed region is bracketed by barriers and the slowest rank's time is used.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import (  # noqa: E402
    config1_plain, config2_ring, config3_fourier, config3_samples, config4_batch, config5_rings)

PARAMS = dict(far_ratio=2.0, tet_gauss_order=4, n_theta=8, n_phi=16)
METRIC = "node-tet interactions/s (velocity at all nodes, FP32 path)"
UNIT = "interactions/s"
# algorithmic FP32 flops (far pair: 8 classify + 4 x 25 quadrature-point; near pair: 8 classify;
# line hit (a chord of a near tet): 80)
FLOPS_FAR_PAIR = 108
FLOPS_NEAR_PAIR_BASE = 8
FLOPS_PER_HIT = 80
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "velocity_fp32_fourier64_traffic.json")
# the device code of the velocity kernel (a stored DRAM-traffic figure applies while these are unchanged and the
# variant's launch shape is the one it was taken with)
KERNEL_SOURCES = [os.path.join(ROOT, "paper_0712_1695_gb300", "csrc", f)
                  for f in ("bs_velocity_kernel.cuh", "bs_near.cuh", "bs_exact.cuh")]


def workload_config():
    return {"workload": "fourier-64^3: 262144 nodes x 1500282 tets, velocity at all nodes",
            "far_ratio": PARAMS["far_ratio"], "tet_gauss_order": PARAMS["tet_gauss_order"],
            "n_theta": PARAMS["n_theta"], "n_phi": PARAMS["n_phi"], "precision": "fp32",
            "l2": "inputs larger than L2 (far records 264 MB, near records 360 MB per replica)"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest of the ranks' values (all-reduce MAX; NCCL wants a device tensor, gloo a host one)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units per second of the whole job: every rank processes units_per_rank (one replica of the
    workload each, weak scaling), the job takes as long as its slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3)


def run_oracle_sample(mesh, count: int, seed_offset: int = 0):
    import oracle

    idx = config3_samples(mesh.n_nodes, 4096)
    rng = np.random.default_rng(77 + seed_offset)
    sel = np.sort(rng.choice(idx, size=count, replace=False))
    t = time.perf_counter()
    v = oracle.velocity(mesh.nodes, mesh.tets, mesh.omega, mesh.nodes[sel], far_ratio=PARAMS["far_ratio"],
                        tet_order=PARAMS["tet_gauss_order"], n_theta=PARAMS["n_theta"], n_phi=PARAMS["n_phi"])
    dt = time.perf_counter() - t
    run_oracle_sample.last = (sel, v)
    return count * mesh.n_tets / dt, dt, oracle.num_threads()


def rms_over_max(v, ref):
    """RMS error over the largest reference speed."""
    return float(np.sqrt(np.mean(np.sum((v - ref) ** 2, axis=1))) / np.linalg.norm(ref, axis=1).max())


def rel_l2(v, ref):
    return float(np.linalg.norm(v - ref) / np.linalg.norm(ref))


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    mesh = config3_fourier()
    import oracle

    oracle.build()
    count = args.ref_sample
    for w in range(args.warmup):
        run_oracle_sample(mesh, max(8, count // 8), seed_offset=100 + w)
    vals, times = [], []
    cores = 1
    for s in range(args.steps):
        v, dt, cores = run_oracle_sample(mesh, count, seed_offset=s)
        vals.append(v)
        times.append(dt)
    value = count * mesh.n_tets * len(times) / sum(times)
    sample = f"{count} of the 4096 seeded sample nodes x all {mesh.n_tets} tets per step (FP64 oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batch_workload(args):
    """256 independent Kuhn meshes (n ~ U{8..24}) with Gaussian blobs: one batched launch (CUDA graph)
    against 256 separate bs_velocity calls, FP32, evaluation points = each mesh's nodes."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    meshes = config4_batch(count=args.batch_count)
    hs = [bs.Mesh(m.nodes, m.tets, m.omega) for m in meshes]
    pairs = sum(m.n_nodes * m.n_tets for m in meshes)
    stream = torch.cuda.Stream()
    P = dict(PARAMS, precision=bs.BS_FP32)
    pts = [torch.from_numpy(m.nodes).cuda() for m in meshes]
    outs_sep = [torch.empty_like(t) for t in pts]
    outs_bat = [torch.empty_like(t) for t in pts]
    batch = bs.Batch(hs)

    def separate():
        for h, t, o in zip(hs, pts, outs_sep):
            h.bs_velocity(t, out_dev=o, stream=stream, **P)

    def batched():
        batch.bs_batch_velocity(outs_bat, stream=stream, **P)

    def timeit(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(steps):
                fn()
            ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    ms_sep = timeit(separate, args.steps) if not args.batch_only else float("nan")
    with ClockSampler(0) as clk:
        ms_bat = timeit(batched, args.steps)
    # accuracy of the FP32 batch against the FP64 path (which is checked against the oracle in the tests)
    outs64 = [torch.empty_like(t) for t in pts]
    with torch.cuda.stream(stream):
        batch.bs_batch_velocity(outs64, stream=stream, **dict(PARAMS, precision=bs.BS_FP64))
        batched()
    torch.cuda.synchronize()
    errs = []
    for a, b in zip(outs_bat, outs64):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        errs.append(np.linalg.norm(a - b) / (np.sqrt(len(b)) * np.linalg.norm(b, axis=1).max()))
    line = {"metric": f"node-tet interactions/s ({len(meshes)}-mesh batch, FP32 path)", "value": pairs / (ms_bat * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_bat,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(meshes)} Kuhn meshes n~U{{8..24}}, Gaussian blobs, {pairs} node-tet pairs",
                       **{k: v for k, v in PARAMS.items()}, "precision": "fp32"},
            "separate_launches": {"ms_per_step": ms_sep, "value": pairs / (ms_sep * 1e-3)},
            "batched_over_separate": ms_sep / ms_bat,
            "fp32_vs_fp64_rms_over_max": {"max": float(max(errs)), "median": float(np.median(errs))},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def rings_workload(args):
    """Two colliding rings on the 80^3 grid: Heun steps (two velocity evaluations at all 512000 nodes
    over 2958234 tets each), FP32; optional drift against an FP64 trajectory on a smaller grid."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    m = config5_rings(n=args.rings_n)
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    stretch = args.rings_mode == "allray-stretch"
    # allray-stretch: the all-ray method (mesh walk) with the vortex-stretching term in the Heun step
    base = dict(PARAMS, far_ratio=float("inf")) if stretch else dict(PARAMS)
    P = dict(base, precision=bs.BS_FP32)

    def step(hh, **kw):
        (hh.bs_rk2_step_stretch if stretch else hh.bs_rk2_step)(0.01, **kw)

    stream = torch.cuda.current_stream()
    for _ in range(min(args.warmup, 1)):  # one warm-up step (a full step is seconds long)
        step(h, **P)
    h.bs_status()
    h = bs.Mesh(m.nodes, m.tets, m.omega)  # start the timed trajectory from t = 0
    # the mesh walk's connectivity (built once per mesh, on the host) and the tables, outside the timed region;
    # its wall time (one evaluation included) and that of a second call give the one-time cost
    first = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.bs_velocity_nodes(**P)
        h.bs_status()
        first.append((time.perf_counter() - t0) * 1e3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(h, **P)
        ev1.record(stream)
        torch.cuda.synchronize()
    h.bs_status()
    ms = ev0.elapsed_time(ev1) / args.steps
    pairs_per_step = 2 * m.n_nodes * m.n_tets
    x = h.bs_nodes().cpu().numpy()
    # drift of the FP32 trajectory against the FP64 one: 20 Heun steps (t = 0.2) on a smaller grid (the FP64
    # trajectory of the 80^3 grid would take hours at the FP64 rate)
    drift = None
    if args.rings_drift_n > 0:
        md = config5_rings(n=args.rings_drift_n)
        traj = {}
        for prec in (bs.BS_FP64, bs.BS_FP32):
            hd = bs.Mesh(md.nodes, md.tets, md.omega)
            for _ in range(20):
                step(hd, **dict(base, precision=prec))
            hd.bs_status()
            traj[prec] = hd.bs_nodes().cpu().numpy()
        dd = np.linalg.norm(traj[bs.BS_FP32] - traj[bs.BS_FP64], axis=1)
        drift = {"grid": f"{args.rings_drift_n}^3", "steps": 20, "dt": 0.01, "max": float(dd.max()),
                 "rms": float(np.sqrt(np.mean(dd ** 2))),
                 "max_displacement_fp64": float(np.abs(traj[bs.BS_FP64] - md.nodes).max())}
    w_change = float(np.abs(h.bs_omega().cpu().numpy() - m.omega).max()) if stretch else 0.0
    line = {"metric": "node-tet interactions/s (RK2 steps of two colliding rings, FP32 path)"
                      + (", all-ray with vortex stretching" if stretch else ""),
            "value": pairs_per_step / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"two rings {args.rings_n}^3: {m.n_nodes} nodes, {m.n_tets} tets, Heun dt=0.01",
                       **{k: (str(v) if k == "far_ratio" else v) for k, v in base.items()}, "precision": "fp32",
                       "mode": args.rings_mode},
            "max_displacement": float(np.abs(x - m.nodes).max()), "max_vorticity_change": w_change,
            "setup_ms": {"first_nodes_call": first[0], "second_nodes_call": first[1]},
            "fp32_vs_fp64_drift": drift,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def allray_workload(args):
    """All-ray evaluation (far_ratio = inf: the ray rule for every pair, the paper's own method) on the
    32^3 Gaussian-ring mesh, velocity at all 32768 nodes, 8x16 directions, FP32: bs_velocity_nodes (lines
    traced through face neighbours), against the all-ray kernel (direction windows) and the velocity
    kernel's dense all-ray path.  With --points, a seeded subset of the nodes through the all-ray kernel
    only (profiling case)."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    big = args.allray_mesh == "fourier64"  # the headline mesh: the walk alone (the other paths take minutes)
    m = config3_fourier() if big else config2_ring()
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    P = dict(PARAMS, far_ratio=float("inf"), precision=bs.BS_FP32)
    L = P["n_theta"] * P["n_phi"]
    nodes = m.nodes
    if args.points:  # a seeded subset of the nodes (small case for profiler captures)
        nodes = m.nodes[np.sort(np.random.default_rng(2002).permutation(m.n_nodes)[:args.points])]
    pairs = len(nodes) * m.n_tets
    stream = torch.cuda.current_stream()
    pts = torch.from_numpy(nodes).cuda()
    out = torch.empty_like(pts)

    def timeit(steps, fn, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        h.bs_status()
        return ev0.elapsed_time(ev1) / steps

    def ray():
        h.bs_velocity(pts, out_dev=out, **P)

    def walk():
        h.bs_velocity_nodes(out_dev=out, **P)

    os.environ["BS_ALLRAY_GENERIC"] = "0"
    ms_walk = ms_ray = ms_dense = None
    v32 = None
    if not args.points:
        with ClockSampler(0) as clk:
            ms_walk = timeit(args.steps, walk, args.warmup)
        v_walk = out.cpu().numpy()
        if not big:
            ms_ray = timeit(args.steps, ray, 1)
    else:
        with ClockSampler(0) as clk:
            ms_ray = timeit(args.steps, ray, args.warmup)
    if ms_ray is not None:
        v32 = out.cpu().numpy()
        os.environ["BS_ALLRAY_GENERIC"] = "1"
        ms_dense = timeit(1, ray, 1)
        os.environ["BS_ALLRAY_GENERIC"] = "0"
    # FP32 against the FP64 all-ray kernel on 512 seeded nodes
    idx = np.random.default_rng(2002).choice(len(nodes), size=min(512, len(nodes)), replace=False)
    v64 = h.bs_velocity(torch.from_numpy(nodes[idx]).cuda(), **dict(P, precision=bs.BS_FP64)).cpu().numpy()
    h.bs_status()

    def err(v):
        return float(np.linalg.norm(v[idx] - v64) / (np.sqrt(len(idx)) * np.linalg.norm(v64, axis=1).max()))

    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        sel = idx[:32] if big else idx[:256]
        t = time.perf_counter()
        oracle.velocity(m.nodes, m.tets, m.omega, nodes[sel], far_ratio=float("inf"),
                        tet_order=PARAMS["tet_gauss_order"], n_theta=PARAMS["n_theta"], n_phi=PARAMS["n_phi"])
        dt = time.perf_counter() - t
        cpu = {"value": len(sel) * m.n_tets / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{len(sel)} seeded nodes x all {m.n_tets} tets, all-ray ({dt:.1f} s)"}
    ms = ms_walk if ms_walk is not None else ms_ray
    line = {"metric": "node-tet interactions/s (all-ray: ray rule for every pair, FP32 path)",
            "value": pairs / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": (f"fourier-64^3: {len(nodes)} nodes x {m.n_tets} tets" if big else
                                    f"gaussian ring 32^3: {len(nodes)} of {m.n_nodes} nodes x {m.n_tets} tets"),
                       **dict(PARAMS, far_ratio="inf"), "precision": "fp32",
                       "path": "mesh walk (bs_velocity_nodes)" if ms_walk is not None else "all-ray kernel"},
            "line_tests_per_s_dense_equivalent": pairs * L / (ms * 1e-3),
            "ray_kernel": None if ms_ray is None else {"ms_per_step": ms_ray, "value": pairs / (ms_ray * 1e-3),
                                                       "fp32_vs_fp64_rms_over_max": err(v32)},
            "dense_loop": None if ms_dense is None else {"ms_per_step": ms_dense, "value": pairs / (ms_dense * 1e-3)},
            "cpu_baseline": cpu, "clocks": clk.summary()}
    if ms_walk is not None:
        line["walk_fp32_vs_fp64_rms_over_max"] = err(v_walk)
        if ms_ray is not None:
            line["walk_over_ray_kernel"] = ms_ray / ms_walk
    print(json.dumps(line), flush=True)
    return 0


def exact_workload(args):
    """The exact near-field rule (the analytic evaluation Section 1 sets the ray rule against) on the 64^3
    Fourier mesh: the hybrid method with ray-rule near pairs (the default) and with exact near pairs, both
    FP32 at all nodes; the extra time per near pair, and the ray rule's error against the exact field on the
    4096 seeded sample nodes (FP64)."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    mesh = config3_fourier()
    h = bs.Mesh(mesh.nodes, mesh.tets, mesh.omega)
    pts = torch.from_numpy(mesh.nodes).cuda()
    out = torch.empty_like(pts)
    cnt = torch.zeros((mesh.n_nodes, 3), dtype=torch.int32, device="cuda")
    res = {}
    with ClockSampler(0) as clk:
        for name, rule in (("ray", bs.BS_NEAR_RAY), ("exact", bs.BS_NEAR_EXACT)):
            P = dict(PARAMS, precision=bs.BS_FP32, near_rule=rule)
            h.bs_velocity(pts, out_dev=out, counts_dev=cnt, **P)
            h.bs_status()
            n_near = int(cnt[:, 0].to(torch.int64).sum())
            for _ in range(max(1, args.warmup - 1)):
                h.bs_velocity(pts, out_dev=out, **P)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                h.bs_velocity(pts, out_dev=out, **P)
            e1.record()
            torch.cuda.synchronize()
            h.bs_status()
            res[name] = {"ms": e0.elapsed_time(e1) / args.steps, "near_pairs": n_near}
    idx = config3_samples(mesh.n_nodes, 4096)
    ps = torch.from_numpy(np.ascontiguousarray(mesh.nodes[idx])).cuda()
    v = {}
    for name, rule in (("ray", bs.BS_NEAR_RAY), ("exact", bs.BS_NEAR_EXACT)):
        v[name] = h.bs_velocity(ps, precision=bs.BS_FP64, **dict(PARAMS, near_rule=rule)).cpu().numpy()
    h.bs_status()
    # the ray rule's cost and error (against the exact rule, FP64 on the samples) as the angular order grows
    sweep = []
    for nt, nphi in ((8, 16), (16, 16), (32, 32), (64, 64)):
        P = dict(PARAMS, n_theta=nt, n_phi=nphi, precision=bs.BS_FP32)
        h.bs_velocity(pts, out_dev=out, **P)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h.bs_velocity(pts, out_dev=out, **P)
        e1.record()
        torch.cuda.synchronize()
        vr = h.bs_velocity(ps, **dict(P, precision=bs.BS_FP64)).cpu().numpy()
        h.bs_status()
        sweep.append({"directions": f"{nphi}x{nt}", "fp32_ms_all_nodes": e0.elapsed_time(e1),
                      "rel_l2_vs_exact": rel_l2(vr, v["exact"])})
    pairs = mesh.n_nodes * mesh.n_tets
    extra = res["exact"]["ms"] - res["ray"]["ms"]
    line = {"metric": "velocity at all nodes with exact near pairs (the analytic near field), FP32 far field",
            "value": pairs / (res["exact"]["ms"] * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["exact"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config(), near_rule="exact"),
            "ray_near_rule": res["ray"], "exact_near_rule": res["exact"],
            "exact_extra_ns_per_near_pair": extra * 1e6 / max(res["exact"]["near_pairs"], 1),
            "ray_vs_exact_fp64": {"rel_l2": rel_l2(v["ray"], v["exact"]),
                                  "rms_over_max": rms_over_max(v["ray"], v["exact"])},
            "ray_rule_by_directions": sweep,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def steps_workload(args):
    """The stage driver on small meshes, where launches dominate: time per Heun step (FP32, far/near rule) of
    bs_rk2_step called per step against bs_rk2_steps (one captured CUDA graph replayed), on the 9^3 plain cube
    and a 16^3 two-ring grid; and the all-ray step with stretching on the plain cube."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    n = max(args.steps, 20)
    rows = []
    cases = [("plain cube 9^3 (729 nodes, 3072 tets), far/near", config1_plain(), dict(PARAMS), False),
             ("two rings 16^3 (4096 nodes, 20250 tets), far/near", config5_rings(n=16), dict(PARAMS), False),
             ("plain cube 9^3, all-ray with stretching (4x8 directions)", config1_plain(),
              dict(far_ratio=float("inf"), tet_gauss_order=4, n_theta=4, n_phi=8), True)]
    with ClockSampler(0) as clk:
        for name, m, P, stretch in cases:
            P = dict(P, precision=bs.BS_FP32)
            res = {}
            for mode in ("eager", "graph"):
                h = bs.Mesh(m.nodes, m.tets, m.omega)
                step = h.bs_rk2_step_stretch if stretch else h.bs_rk2_step
                for _ in range(3):  # warm-up: connectivity, tables, work arrays
                    step(0.001, **P)
                h.bs_status()
                t0 = time.perf_counter()
                if mode == "eager":
                    for _ in range(n):
                        step(0.001, **P)
                else:
                    h.bs_rk2_steps(0.001, n, stretch=stretch, **P)
                torch.cuda.synchronize()
                res[mode] = 1e3 * (time.perf_counter() - t0) / n
                h.bs_status()
                if mode == "graph":
                    res["graph_steps"] = h.bs_graph_steps()
            rows.append({"case": name, "steps": n, "eager_ms_per_step": res["eager"],
                         "graph_ms_per_step": res["graph"], "speedup": res["eager"] / res["graph"],
                         "graph_replays": res["graph_steps"]})
    line = {"metric": "Heun step time on small meshes, per-step calls vs one replayed CUDA graph", "unit": "ms",
            "higher_is_better": False, "rows": rows, "clocks": clk.summary(),
            "note": "wall clock over the steps after the device work is done (the host enqueue cost included)"}
    print(json.dumps(line), flush=True)
    return 0


def variants_workload(args):
    """Every variant of the float32 four-point ray rule on the headline workload (the 64^3 Fourier mesh at
    all nodes, or --points nodes nearest the centre), each pinned in turn: ms per evaluation (mean of
    --steps after --warmup) and the shape.  The nodes are evaluated as arbitrary points (bs_velocity: far sweep
    and near pass or in-kernel drain), or with --at-nodes by bs_velocity_nodes (the walk takes the near field of
    the variants that leave it out)."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    mesh = config3_fourier()
    h = bs.Mesh(mesh.nodes, mesh.tets, mesh.omega)
    nodes = mesh.nodes
    if args.points:
        sel = np.sort(np.argsort(np.linalg.norm(mesh.nodes, axis=1), kind="stable")[:args.points])
        nodes = np.ascontiguousarray(mesh.nodes[sel])
    if args.at_nodes and args.points:
        raise SystemExit("--at-nodes evaluates all nodes; drop --points")
    pts = torch.from_numpy(nodes).cuda()
    out = torch.empty_like(pts)
    P = dict(PARAMS, precision=bs.BS_FP32)
    n = bs.bs_num_variants(bs.BS_FP32, 4)
    only = [int(v) for v in args.variants.split(",")] if args.variants else range(n)
    rows = []
    with ClockSampler(0) as clk:
        for v in only:
            h.bs_set_variant(bs.BS_FP32, 4, bs.BS_NEAR_RAY, v)

            def run():
                if args.at_nodes:
                    h.bs_velocity_nodes(out_dev=out, **P)
                else:
                    h.bs_velocity(pts, out_dev=out, **P)
            for _ in range(args.warmup):
                run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                run()
            e1.record()
            torch.cuda.synchronize()
            h.bs_status()
            ms = e0.elapsed_time(e1) / args.steps
            rows.append(dict(bs.bs_variant_shape(bs.BS_FP32, 4, bs.BS_NEAR_RAY, v), variant=v, ms=ms,
                             interactions_per_s=len(nodes) * mesh.n_tets / (ms * 1e-3)))
    rows.sort(key=lambda r: r["ms"])
    print(json.dumps({"metric": "ms per evaluation by kernel variant (FP32, 4-point rule, 8x16 directions)",
                      "path": "bs_velocity_nodes" if args.at_nodes else "bs_velocity",
                      "points": len(nodes), "tets": mesh.n_tets, "steps": args.steps, "warmup": args.warmup,
                      "rows": rows, "clocks": clk.summary()}), flush=True)
    return 0


def rules_workload(args):
    """At the nodes of the 24^3 two-ring mesh (bs_velocity_nodes, 8x16 directions), for each precision and tet
    rule: variant 0 pinned, the first variant that leaves the near pairs to the mesh walk pinned, and the
    library's own choice without a pin (ms per evaluation, mean of --steps after --warmup) and the RMS
    difference over max speed of each against variant 0."""
    import torch

    import paper_0712_1695_gb300 as bs

    bs.load()
    m = config5_rings(24)
    h = bs.Mesh(m.nodes, m.tets, m.omega)
    rows = []
    with ClockSampler(0) as clk:
        for prec, pname in ((bs.BS_FP32, "fp32"), (bs.BS_FP64, "fp64")):
            for q in (1, 4, 8, 27, 64):
                P = dict(PARAMS, tet_gauss_order=q, precision=prec)
                nv = bs.bs_num_variants(prec, q)
                walk = [v for v in range(nv) if bs.bs_variant_shape(prec, q, bs.BS_NEAR_RAY, v)["near_drain"] == 3]
                ref = None
                for label, v in (("variant 0", 0), ("near pairs to the walk", walk[0]), ("unpinned", -1)):
                    h.bs_set_variant(prec, q, bs.BS_NEAR_RAY, v)
                    for _ in range(max(args.warmup, 1)):
                        o = h.bs_velocity_nodes(**P)
                    torch.cuda.synchronize()
                    h.bs_status()
                    if ref is None:
                        ref = o.clone()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(args.steps):
                        h.bs_velocity_nodes(**P)
                    e1.record()
                    torch.cuda.synchronize()
                    h.bs_status()
                    d = float(torch.sqrt(((o - ref) ** 2).sum(1).mean()) / ref.norm(dim=1).max())
                    rows.append({"precision": pname, "tet_rule": q, "choice": label, "variant": v,
                                 "ms": e0.elapsed_time(e1) / args.steps, "rms_over_max_vs_variant0": d})
                h.bs_set_variant(prec, q, bs.BS_NEAR_RAY, -1)
    print(json.dumps({"metric": "ms per evaluation at all nodes by variant choice (two rings 24^3: "
                                f"{m.n_nodes} nodes x {m.n_tets} tets, far_ratio 2, 8x16 directions)",
                      "steps": args.steps, "warmup": args.warmup, "rows": rows, "clocks": clk.summary()}),
          flush=True)
    return 0


def fma_probe():
    """The bench-only fma-chain probe (bench_fma_probe.cu), compiled on demand with the library's nvcc flags."""
    import ctypes

    from paper_0712_1695_gb300.build import ARCH, nvcc

    src = os.path.join(ROOT, "bench_fma_probe.cu")
    lib = os.path.join(ROOT, "_build", "libfma_probe.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(lib), exist_ok=True)
        subprocess.run([nvcc(), *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", src, "-o", lib], check=True)
    so = ctypes.CDLL(lib)
    so.fma_probe_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]

    def rate(kind):
        r = ctypes.c_double()
        if so.fma_probe_rate(kind, ctypes.byref(r)) != 0:
            raise RuntimeError(f"fma probe kind {kind} failed")
        return r.value

    return rate


def peaks_workload(args):
    """Measured arithmetic rates of this GPU (bench_fma_probe.cu): float64 fma (the float64 path and the exact
    near rule), float32 fma and packed float32x2 fma (the far sweep), beside the nominal float32 peak the
    headline's roofline divides by."""
    import torch

    rate = fma_probe()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    with ClockSampler(0) as clk:
        rates = {name: max(rate(kind) for _ in range(2))
                 for name, kind in (("fp64_fma", 0), ("fp32_fma", 1), ("fp32x2_fma", 2))}
    nominal = n_sm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
    line = {"metric": "measured fma-chain rates", "unit": "TFLOP/s", "rates": rates,
            "fp32_nominal_peak": nominal, "fp32x2_over_nominal": rates["fp32x2_fma"] / nominal,
            "fp64_over_fp32": rates["fp64_fma"] / rates["fp32_fma"], "n_sm": n_sm, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fourier64",
                    choices=["fourier64", "batch", "rings", "allray", "exact", "peaks", "steps", "variants", "rules"],
                    help="fourier64: the headline workload; batch: 256 uneven meshes, batched vs separate "
                         "launches; rings: Heun steps of two colliding rings; allray: the ray rule for every "
                         "pair on the 32^3 ring mesh; "
                         "exact: the exact near-field rule against the ray rule on the 64^3 mesh; peaks: measured fma rates; "
                         "steps: Heun steps on small meshes, per-step calls vs a replayed CUDA graph; variants: "
                         "every float32 kernel variant timed on the headline workload; rules: at the nodes of a "
                         "24^3 mesh, variant 0 against the variant leaving the near pairs to the walk, per precision "
                         "and tet rule")
    ap.add_argument("--at-nodes", action="store_true",
                    help="variants workload: evaluate through bs_velocity_nodes (all nodes only)")
    ap.add_argument("--rings-n", type=int, default=80, help="nodes per side of the rings workload")
    ap.add_argument("--rings-mode", default="hybrid", choices=["hybrid", "allray-stretch"],
                    help="rings workload: the far/near rule with frozen vorticity, or the all-ray method with vortex "
                         "stretching")
    ap.add_argument("--rings-drift-n", type=int, default=56,
                    help="rings workload: grid of the FP32-vs-FP64 drift run (20 Heun steps; 0 to skip). The default "
                         "56^3 is the largest grid whose FP64 trajectory takes minutes (about 15 on a GB300); the "
                         "80^3 one would take about 2.2 hours")
    ap.add_argument("--allray-mesh", default="ring32", choices=["ring32", "fourier64"],
                    help="allray workload: the 32^3 ring mesh (walk, all-ray kernel, dense path) or the 64^3 "
                         "Fourier mesh (the walk alone)")
    ap.add_argument("--batch-count", type=int, default=256, help="meshes in the batch workload")
    ap.add_argument("--batch-only", action="store_true", help="batch workload: skip the separate-launch timing")
    ap.add_argument("--cpu-sample", type=int, default=640, help="oracle sample nodes for cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=96, help="oracle sample nodes per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 path on the 4096 sample nodes")
    ap.add_argument("--variants", default="", help="variants workload: comma-separated variant indices (default all)")
    ap.add_argument("--grid", type=int, default=64,
                    help="nodes per side of the Fourier workload (64: the headline; smaller grids are profiling cases)")
    ap.add_argument("--points", type=int, default=0,
                    help="evaluate only this many seeded nodes (small case for profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "batch":
        return batch_workload(args)
    if args.workload == "rings":
        return rings_workload(args)
    if args.workload == "allray":
        return allray_workload(args)
    if args.workload == "exact":
        return exact_workload(args)
    if args.workload == "peaks":
        return peaks_workload(args)
    if args.workload == "steps":
        return steps_workload(args)
    if args.workload == "variants":
        return variants_workload(args)
    if args.workload == "rules":
        return rules_workload(args)

    import torch

    import paper_0712_1695_gb300 as bs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    bs.load()
    mesh = config3_fourier(args.grid)
    h = bs.Mesh(mesh.nodes, mesh.tets, mesh.omega)
    eval_nodes = mesh.nodes
    if args.points:
        # a compact patch (the nodes nearest the centre): warps see the same culling as on the full grid
        sel = np.sort(np.argsort(np.linalg.norm(mesh.nodes, axis=1), kind="stable")[:args.points])
        eval_nodes = np.ascontiguousarray(mesh.nodes[sel])
    k = len(eval_nodes)
    pairs = k * mesh.n_tets
    stream = torch.cuda.current_stream()
    pts = torch.from_numpy(eval_nodes).cuda()
    out = torch.empty((k, 3), dtype=torch.float64, device="cuda")
    P = dict(PARAMS, precision=bs.BS_FP32)
    at_nodes = not args.points  # the velocity at the mesh's own nodes: bs_velocity_nodes

    def evaluate(counts=None):
        if at_nodes:
            h.bs_velocity_nodes(out_dev=out, counts_dev=counts, **P)
        else:
            h.bs_velocity(pts, out_dev=out, counts_dev=counts, **P)

    # the kernel variant: the autotuner's choice for this GPU and workload (a hit in the shipped tuning
    # cache on a GB300; timed once otherwise)
    if os.environ.get("BS_VARIANT"):  # pinned for every call: nothing to tune
        variant, chosen_by = int(os.environ["BS_VARIANT"]), "BS_VARIANT"
    else:
        h.bs_autotune(**P)
        variant, chosen_by = h.bs_tuned_variant(bs.BS_FP32, PARAMS["tet_gauss_order"], at_nodes), "bs_autotune"
    variant_shape = bs.bs_variant_shape(bs.BS_FP32, PARAMS["tet_gauss_order"], bs.BS_NEAR_RAY, variant)

    # counts of one untimed evaluation give the algorithmic flops of a launch: the far rule's per pair, the
    # near/far test per near pair and the chord integral per line hit (the work that makes the result)
    cnt = torch.zeros((k, 3), dtype=torch.int32, device="cuda")
    evaluate(cnt)
    h.bs_status()
    c = cnt.to(torch.int64).sum(dim=0).cpu().numpy()
    n_near, n_far, n_hit = int(c[0]), int(c[1]), int(c[2])
    flops = n_far * FLOPS_FAR_PAIR + n_near * FLOPS_NEAR_PAIR_BASE + n_hit * FLOPS_PER_HIT

    for _ in range(args.warmup):
        evaluate()
    barrier()

    # the timed region: the production path (no profiling events), inputs resident in HBM
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            evaluate()
        ev1.record(stream)
        barrier()
    h.bs_status()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(pairs, world, ms_max)

    # a separate profiled pass (untimed for `value`): the velocity kernel's own event time on its launch
    # stream, and the number of the library's kernel launches per step
    prof_steps = max(1, min(args.steps, 3))
    h.bs_profile(True)
    for _ in range(prof_steps):
        evaluate()
    kernel_ms, kernel_launches, all_launches = h.bs_profile_read()
    h.bs_profile(False)
    h.bs_status()
    launches_per_step = all_launches / prof_steps

    # end to end through the public C ABI, every step: the step's node positions and vorticity copied from
    # pinned host memory to the device and bs_update (a Lagrangian step's new mesh), bs_velocity_nodes, and
    # the velocities copied back to pinned host memory
    nodes_h = torch.from_numpy(mesh.nodes).pin_memory()
    omega_h = torch.from_numpy(mesh.omega).pin_memory()
    vel_h = torch.empty((k, 3), dtype=torch.float64).pin_memory()
    nodes_d = torch.empty((mesh.n_nodes, 3), dtype=torch.float64, device="cuda")
    omega_d = torch.empty_like(nodes_d)

    def e2e_step():
        nodes_d.copy_(nodes_h, non_blocking=True)
        omega_d.copy_(omega_h, non_blocking=True)
        h.bs_update(nodes_d, omega_d)
        h.bs_velocity_nodes(out_dev=out, **P)
        vel_h.copy_(out, non_blocking=True)
        stream.synchronize()

    e2e = None
    if not args.no_e2e and not args.points:
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": whole_job_rate(pairs, world, 1e3 * max_over_ranks(e2e_s, dist, "cuda")), "unit": UNIT,
               "h2d_bytes_per_step": 2 * mesh.n_nodes * 24, "d2h_bytes_per_step": k * 24,
               "ms_per_step": 1e3 * e2e_s}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(local_rank)
    n_sm = props.multi_processor_count
    clocks = clk.summary()
    kernel_avg_ms = kernel_ms / max(kernel_launches, 1)
    achieved = flops / (kernel_avg_ms * 1e-3) / 1e12
    peak = n_sm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
    traffic = None
    if os.path.exists(PROFILE_TRAFFIC):
        with open(PROFILE_TRAFFIC) as f:
            tr = json.load(f)
        shape = "P{points_per_thread} T{tile} S{stages} B{ctas_per_sm} D{near_drain} U{ray_bundle} {pk} J{tet_unroll}".format(
            pk="pp" if variant_shape["point_pairs"] else "qp", **variant_shape)
        if tr.get("kernel_source_hash") == kernel_source_hash() and tr.get("shape") == shape:
            traffic = tr.get("dram_bytes_per_launch")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic,
                "kernel": "velocity_kernel (float, 4-point far rule)" + (
                    " + near field (" + ("mesh walk" if at_nodes else "near pass") + ")"
                    if variant_shape["near_drain"] == 3 else ", near pairs drained in the kernel"),
                "kernel_ms": kernel_avg_ms,
                "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {MAX_SM_MHZ:.0f} MHz",
                "flops_per_launch": flops}
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (n_sm * FP32_LANES_PER_SM * 2 * clocks["sm_mhz"] * 1e-6)

    # the FP64 path on the 4096 seeded sample nodes: its rate and the FP32 path's error against it
    fp64 = None
    v32 = out.cpu().numpy()
    if not args.no_fp64 and not args.points:
        idx = config3_samples(mesh.n_nodes, 4096)
        pts64 = torch.from_numpy(np.ascontiguousarray(mesh.nodes[idx])).cuda()
        out64 = torch.empty((len(idx), 3), dtype=torch.float64, device="cuda")
        P64 = dict(PARAMS, precision=bs.BS_FP64)
        h.bs_velocity(pts64, out_dev=out64, **P64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.bs_velocity(pts64, out_dev=out64, **P64)
        e1.record(stream)
        torch.cuda.synchronize()
        h.bs_status()
        v64 = out64.cpu().numpy()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": len(idx) * mesh.n_tets / (ms64 * 1e-3), "unit": UNIT, "ms": ms64,
                "sample": f"the 4096 seeded sample nodes x all {mesh.n_tets} tets",
                "fp32_vs_fp64_rms_over_max": rms_over_max(v32[idx], v64),
                "fp32_vs_fp64_rel_l2": rel_l2(v32[idx], v64)}

    cpu = None
    if not args.no_cpu_baseline and world == 1 and not args.points:
        import oracle

        oracle.build()
        run_oracle_sample(mesh, 8, seed_offset=999)  # page in
        v, dt, cores = run_oracle_sample(mesh, args.cpu_sample)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} of the 4096 seeded sample nodes x all {mesh.n_tets} tets ({dt:.1f} s)"}
        sel, vo = run_oracle_sample.last
        # one core, on a smaller sample of the same nodes
        all_threads = oracle.num_threads()
        oracle.set_num_threads(1)
        v1, dt1, _ = run_oracle_sample(mesh, 48, seed_offset=7)
        oracle.set_num_threads(all_threads)
        cpu["one_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                           "sample": f"48 of the 4096 seeded sample nodes x all {mesh.n_tets} tets ({dt1:.1f} s)"}
        cpu["fp32_vs_oracle_rms_over_max"] = rms_over_max(v32[sel], vo)
        cpu["fp32_vs_oracle_rel_l2"] = rel_l2(v32[sel], vo)
        if fp64 is not None:
            pos = np.searchsorted(idx, sel)
            if np.array_equal(idx[pos], sel):
                cpu["fp64_vs_oracle_rel_l2"] = rel_l2(v64[pos], vo)

    config = workload_config()
    if args.points:
        config["workload"] = (f"fourier-{args.grid}^3 mesh ({mesh.n_tets} tets), velocity at the {k} nodes nearest the "
                              "centre (profiling case)")
    elif args.grid != 64:
        config["workload"] = (f"fourier-{args.grid}^3: {mesh.n_nodes} nodes x {mesh.n_tets} tets, velocity at all nodes "
                              "(profiling case)")
    if args.grid != 64:  # far records 176 B and near records 240 B per tet (float32 + float64 copies)
        far_mb, near_mb = mesh.n_tets * 176 / 1e6, mesh.n_tets * 240 / 1e6
        config["l2"] = (f"far records {far_mb:.0f} MB, near records {near_mb:.0f} MB: "
                        + ("larger than L2" if far_mb > 129 else "the far records fit in L2"))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
            "roofline": roofline, "cpu_baseline": cpu, "fp64_path": fp64,
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)), "clocks": clocks,
            "variant": dict(variant_shape, index=variant, chosen_by=chosen_by),
            "counts": {"near_pairs": n_near, "far_pairs": n_far, "ray_hits": n_hit}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
