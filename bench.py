#!/usr/bin/env python
"""Benchmark of the exact mesh-to-grid projection on GB300.

Metric: tetrahedra projected per second on a 256^3 grid (FP32-mixed path; the FP64 path is timed
beside it in the same run). Workload (synthetic, seeded): a 128^3 Lagrangian lattice of Kuhn cubes
(12,582,912 tetrahedra, 2,097,152 vertices) displaced by a curl-free Gaussian random field with
power spectrum k^-2 for |k| <= 16 and rms 4 Lagrangian cells (post shell-crossing), lognormal
vertex density (sigma = 0.5), periodic unit box, 256^3 FP64 output grid.

One step = one full projection: zeroing the grid, vertex records, the per-tetrahedron set-up, the
block-cooperative projection kernel and the tiled large-tetrahedron kernel, all through the C ABI. Inputs (201 MB of simplices, 67 MB of vertex records,
134 MB grid) exceed the 129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank projects its own replica (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c3"
METRIC = "tetrahedra projected/s on 256^3 grid, FP32-mixed vs FP64 plain, same GB300"
UNIT = "tets/s"

# Algorithmic FP32 work of the Franklin evaluation per (corner, cell) incidence: six
# (vertex, edge, facet) triples of 3+3 dot products (5 flops each), the bracket (9) and the triple
# product (3) = 42 flops each; the type-A closed form is 12 flops.
FLOPS_PER_INCIDENCE = {"a": 12, "b": 252, "c": 252, "d": 252}
# DRAM bytes (read + write) of one k_project_tet<float> launch per tetrahedron, from the ncu capture
# summarised in profiles/k_project_tet_c3s64_full.md (1,572,864 tetrahedra: 713.1 MB read, 86.9 MB
# written); the traffic is the geometry records plus the grid atomics, so it scales with the
# tetrahedron count.  None while the kernel has changed since the capture.
TRAFFIC_BYTES_PER_TET = (713.054976e6 + 86.854400e6) / 1572864
# ALU peaks derived from unit counts and the maximum SM clock (no measured FP32 figure exists):
# 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz; FP64 1.25 TFLOP/s nominal.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=None, help="Lagrangian lattice size override (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 plain path")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 64-problem step (c5)")
    return ap.parse_args()


def _batched_step(pkg, mg, proj, dev, stream, steps=3, warmup=3):
    """The batched workload c5: 64 independent 2D/3D problems advanced by one time step each (drift,
    vertex density, FP32-mixed projection, FFT Poisson, force, kick, drift) as one replayed CUDA
    graph.  Inputs resident on the device; CUDA events around the replays."""
    import torch

    batch = mg.make_batch("c5")
    dt = mg.cfl_dt(batch)
    keep = []
    probs = []
    for p in batch:
        m = p.mesh
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        pos = [t(m.pos[a]) for a in range(m.dim)]
        vel = [t(p.vel[a]) for a in range(m.dim)]
        acc = [torch.zeros(m.n_verts, dtype=torch.float64, device=dev) for _ in range(m.dim)]
        simp, mass = t(m.simplices), t(p.masses)
        rho = torch.zeros(m.n_verts, dtype=torch.float64, device=dev)
        cm = torch.zeros(m.grid, dtype=torch.float64, device=dev)
        phi = torch.zeros(m.grid, dtype=torch.float64, device=dev)
        sp = pkg.cdp_step_problem()
        sp.mesh = pkg.Projector.make_problem(pos, simp, rho, m.grid, m.box_lo, m.box_len, True, cm)
        for a in range(m.dim):
            sp.vel[a] = vel[a].data_ptr()
            sp.acc[a] = acc[a].data_ptr()
        sp.simplex_mass = mass.data_ptr()
        sp.phi = phi.data_ptr()
        probs.append(sp)
        keep.append((pos, vel, acc, simp, mass, rho, cm, phi))
    arr = (pkg.cdp_step_problem * len(probs))(*probs)
    st = stream.cuda_stream
    for _ in range(warmup):  # the first call captures the graph
        rc = pkg.cdp_step_batched(proj._ctx, arr, pkg.CDP_FP32_MIXED, dt, 1.0, True, st)
        if rc:
            raise RuntimeError(f"cdp_step_batched: {rc}")
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pkg.cdp_step_batched(proj._ctx, arr, pkg.CDP_FP32_MIXED, dt, 1.0, True, st)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    ns = sum(p.mesh.n_simplices for p in batch)
    del keep
    return {"workload": "c5: 64 problems (32 3D Kuhn/GRF, 32 2D two-sine), simplex counts log-uniform "
                        "in [1e3, 2e6], grids 64..256 per axis; one time step each as one CUDA graph",
            "problems": len(batch), "simplices": ns, "ms_per_step": ms, "simplices_per_s": ns / (ms / 1000.0),
            "dtype": "f32-mixed projection, f64 solver", "steps": steps, "warmup": warmup}


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _cpu_baseline(mesh, target_s=12.0, seed=5):
    """The oracle as it stands, on a random subset of the workload's simplices (host cores)."""
    import oracle

    rng = np.random.default_rng(seed)
    ns = mesh.n_simplices
    n = min(ns, 20000)
    idx = np.sort(rng.choice(ns, n, replace=False))
    t0 = time.perf_counter()
    oracle.project(mesh.subset(idx))
    dt = time.perf_counter() - t0
    rate = n / dt
    n2 = int(min(ns, max(n, rate * target_s)))
    idx = np.sort(rng.choice(ns, n2, replace=False))
    t0 = time.perf_counter()
    oracle.project(mesh.subset(idx))
    dt = time.perf_counter() - t0
    # the same oracle on one thread, on a sample of a few seconds (comparable to a per-thread figure)
    n1 = int(min(ns, max(1000, n2 / max(oracle.max_threads(), 1) / 3)))
    idx1 = np.sort(rng.choice(ns, n1, replace=False))
    t1 = time.perf_counter()
    oracle.project(mesh.subset(idx1), nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": n2 / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n2} of {ns} tetrahedra of the workload, chosen uniformly at random (seed {seed}), "
                      f"projected onto the full 256^3 grid in {dt:.1f} s",
            "one_thread": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                           "sample": f"{n1} random tetrahedra of the workload in {dt1:.1f} s"}}


def max_over_ranks(v: float, ws: int, device) -> float:
    """The largest of the ranks' values of v (an all-reduce MAX on `device`); v itself on one rank."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job units per second: every rank processes units_per_rank in a step, and the step takes
    the slowest rank's ms_max."""
    return ws * units_per_rank / (ms_max / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(a):
    """Reference arm: the CPU oracle timed on this machine's host cores, each step a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1509_07720_gb300 import meshgen as mg

    mesh = mg.make_config(WORKLOAD, a.scale)
    rng = np.random.default_rng(17)
    ns = mesh.n_simplices
    per_step = min(ns, 40000)
    for _ in range(a.warmup):
        oracle.project(mesh.subset(np.sort(rng.choice(ns, min(ns, 2000), replace=False))))
    times = []
    for _ in range(a.steps):
        idx = np.sort(rng.choice(ns, per_step, replace=False))
        sub = mesh.subset(idx)
        t0 = time.perf_counter()
        oracle.project(sub)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * a.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "128^3 Kuhn lattice (12,582,912 tets), GRF k^-2 k<=16 rms 4 cells, lognormal rho "
                               "sigma 0.5, 256^3 grid; each step a random sample of %d tets" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{per_step} random tetrahedra per step of the {ns}-tet workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(a):
    import torch

    import paper_1509_07720_gb300 as pkg
    from paper_1509_07720_gb300 import build, meshgen as mg

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    build.build_library()

    mesh = mg.make_config(WORKLOAD, a.scale)
    ns = mesh.n_simplices
    pos = torch.from_numpy(np.ascontiguousarray(mesh.pos)).to(dev)
    simp = torch.from_numpy(np.ascontiguousarray(mesh.simplices)).to(dev)
    rho = torch.from_numpy(np.ascontiguousarray(mesh.rho)).to(dev)
    out = torch.empty(mesh.grid, dtype=torch.float64, device=dev)
    proj = pkg.Projector(local)
    stream = torch.cuda.current_stream(dev)

    def step(prec):
        proj.project(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, True, precision=prec, out=out,
                     stream=stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    # one instrumented pass for the corner counts (outside every timed region)
    _, st32 = proj.project(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, True,
                           precision=pkg.CDP_FP32_MIXED, out=out, stream=stream, stats=True)

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        proj.timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(prec)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        kern, calls = proj.timing()
        proj.timing(False)
        return ms, [k / max(calls, 1) for k in kern]

    clk = ClockSampler(local)
    clk.start()
    ms32, kern32 = timed(pkg.CDP_FP32_MIXED, a.steps, a.warmup)
    clocks = clk.stop()
    proj.check(stream)
    ms32 = max_over_ranks(ms32, ws, dev)
    value = job_throughput(ws, ns, ms32)

    # FP64 plain path on the same GPU, same workload (fewer steps: it is much slower)
    k64 = max(1, a.fp64_steps)
    ms64, kern64 = timed(pkg.CDP_FP64, k64, 1)
    ms64 = max_over_ranks(ms64, ws, dev)

    # end to end through the C ABI from pinned host buffers: H2D inputs, project, D2H grid
    e2e = None
    if not a.no_e2e:
        hp = torch.from_numpy(np.ascontiguousarray(mesh.pos)).pin_memory()
        hs = torch.from_numpy(np.ascontiguousarray(mesh.simplices)).pin_memory()
        hr = torch.from_numpy(np.ascontiguousarray(mesh.rho)).pin_memory()
        ho = torch.empty(mesh.grid, dtype=torch.float64).pin_memory()
        dpos = torch.empty_like(pos)
        dsimp = torch.empty_like(simp)
        drho = torch.empty_like(rho)

        def e2e_step():
            dpos.copy_(hp, non_blocking=True)
            dsimp.copy_(hs, non_blocking=True)
            drho.copy_(hr, non_blocking=True)
            proj.project(dpos, dsimp, drho, mesh.grid, mesh.box_lo, mesh.box_len, True,
                         precision=pkg.CDP_FP32_MIXED, out=out, stream=stream)
            ho.copy_(out, non_blocking=True)

        for _ in range(a.warmup):
            e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        mse = max_over_ranks(e0.elapsed_time(e1) / a.steps, ws, dev)
        hb = hp.numel() * 8 + hs.numel() * 4 + hr.numel() * 8
        e2e = {"value": job_throughput(ws, ns, mse), "unit": UNIT, "h2d_bytes_per_step": int(hb),
               "d2h_bytes_per_step": int(ho.numel() * 8), "ms_per_step": mse}

    # the batched workload (every rank runs its own replica; rank 0 reports its own)
    batched = None if a.no_batched else _batched_step(pkg, mg, proj, dev, stream)

    if rank != 0:
        return
    # roofline of the dominant kernel (the tetrahedron projection kernel; its incidences are all
    # corners but those found on the tiles of the large tetrahedra, by k_project_big)
    names = ["k_prep_vertices", "k_tet_setup<float>", "k_project_tet<float>", "k_project_big<float>"]
    dom = int(np.argmax(kern32))
    if dom == 2:
        inc = {k: st32["corners_" + k] - st32["large_corners"][i] for i, k in enumerate("abcd")}
    else:
        inc = None
    if inc is not None:
        flops = sum(FLOPS_PER_INCIDENCE[k] * v for k, v in inc.items())
        achieved = flops / (kern32[dom] / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": None if TRAFFIC_BYTES_PER_TET is None else TRAFFIC_BYTES_PER_TET * ns,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                "scale-64 capture scaled by tetrahedra)", "kernel": names[dom],
                "kernel_ms": kern32[dom], "flops_per_launch": flops,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    else:
        hbm = _measured_peaks().get("hbm_gbs", 6800.0)
        byts = mesh.n_verts * (3 * 8 + 8 + 32)
        achieved = byts / (kern32[0] / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": names[0]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-mixed (f64 accumulate)", "data": "synthetic",
        "config": {"workload": "128^3 Kuhn lattice (12,582,912 tets), GRF k^-2 k<=16 rms 4 cells, lognormal rho "
                               "sigma 0.5, periodic, 256^3 FP64 grid" if a.scale is None else f"c3 scale {a.scale}",
                   "tets": ns, "grid": list(mesh.grid), "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{ws}"},
        "fp64_plain": {"value": job_throughput(ws, ns, ms64), "unit": UNIT, "ms_per_step": ms64,
                       "kernel_ms": kern64, "speedup_fp32_mixed_vs_fp64": ms64 / ms32},
        "kernel_ms": dict(zip(names, kern32)),
        "corners": {k: st32[k] for k in ("corners_a", "corners_b", "corners_c", "corners_d", "n_single_cell",
                                         "n_small", "n_large", "n_zero_volume", "exact_fallbacks")},
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": 4 * a.steps,  # vertex records, set-up, main kernel, large tetrahedra (one batch)
        "e2e": e2e,
    }
    if not a.no_batched:
        line["batched"] = batched
    if ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(mesh)
    print(json.dumps(line), flush=True)
    proj.close()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
