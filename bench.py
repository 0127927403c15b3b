#!/usr/bin/env python
"""Benchmark of the exact mesh-to-grid projection on GB300.

Metric: tetrahedra projected per second on a 256^3 grid (FP32-mixed path; the FP64 path is timed
beside it in the same run). Workload (synthetic, seeded): a 128^3 Lagrangian lattice of Kuhn cubes
(12,582,912 tetrahedra, 2,097,152 vertices) displaced by a curl-free Gaussian random field with
power spectrum k^-2 for |k| <= 16 and rms 4 Lagrangian cells (post shell-crossing), lognormal
vertex density (sigma = 0.5), periodic unit box, 256^3 FP64 output grid.

One step = one full projection: zeroing the grid, vertex records, the per-tetrahedron set-up, the
block-cooperative projection kernel and the tiled large-tetrahedron kernel, all through the C ABI.
Inputs (201 MB of simplices, 67 MB of vertex records, 134 MB grid) exceed the 129 MB L2, so no
flush is needed between steps.

``--config`` selects another workload of the same family, each printed as its own JSON line of the
same form (``all``: every one, the headline first):
  c1a / c1b  2D: 64^2 Lagrangian squares (8,192 triangles), two sine waves (single / multi-stream),
             128^2 grid
  c2         3D: 32^3 Kuhn cubes (196,608 tets), GRF rms 0.5 cell, 128^3 grid
  c3         the headline workload above
  c4         3D: a 64^3 Kuhn base bisected to 50,331,953 tets (volumes over four decades), 512^3
             grid
  c5         64 independent 2D/3D problems (18.3M simplices): their projections in one call, and one
             time step of all of them (drift, vertex density, projection, Poisson, force, kick,
             drift) replayed as one CUDA graph

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]
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
CONFIG_CHOICES = ("c3", "c1a", "c1b", "c2", "c4", "c5", "all")

# Algorithmic FP32 work per (corner, cell) incidence of the Franklin evaluation: the upper figure
# of the 100-200 flops a B, C or D incidence takes (six (vertex, edge, facet) triples, each three
# projections of the corner and three of the gradient on its frame, the bracket and the triple
# product), and 12 flops for the closed form of an A incidence (the corner's three offsets, their
# product, the bracket).
FLOPS_PER_INCIDENCE = {"a": 12, "b": 200, "c": 200, "d": 200}
# Per-tetrahedron counters of one k_project_tet<float> launch, from the ncu capture summarised in
# profiles/k_project_tet_c3sub8_full.md (a random 1/8 of the headline workload's tetrahedra,
# 1,572,864, on its own 256^3 grid): DRAM bytes read + written, and warp instructions issued.
# They scale with the tetrahedron count.  None while the kernel has changed since the capture.
TRAFFIC_BYTES_PER_TET = 655.6
WARP_INST_PER_TET = 2738.9


def _args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD, choices=CONFIG_CHOICES)
    ap.add_argument("--scale", type=int, default=None, help="Lagrangian lattice size override (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 plain path")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 64-problem step (c5)")
    ap.add_argument("--amr", type=int, default=None,
                    help="also time the projection through the levels 0..AMR with donor-cell gather (cdp_project_amr); "
                         "default: 3 for the c2 and c4 workloads, none otherwise")
    return ap.parse_args(argv)


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


def _json_file(name):
    try:
        with open(os.path.join(ROOT, name)) as f:
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
            "sample": f"{n2} of {ns} simplices of the workload, chosen uniformly at random (seed {seed}), "
                      f"projected onto the full grid in {dt:.1f} s",
            "one_thread": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                           "sample": f"{n1} random simplices of the workload in {dt1:.1f} s"}}


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


def workload_text(name, mesh=None, scale=None):
    from paper_1509_07720_gb300 import meshgen as mg

    if name == "c5":
        return ("c5: 64 problems (32 3D Kuhn/GRF, 32 2D two-sine), simplex counts log-uniform in [1e3, 2e6], grids "
                "64..256 per axis")
    txt = mg.CONFIG_NAMES[name] + ", periodic, FP64 grid"
    return txt if scale is None else f"{txt} (lattice scale {scale})"


def run_reference(a):
    """Reference arm: the CPU oracle timed on this machine's host cores, each step a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1509_07720_gb300 import meshgen as mg

    name = WORKLOAD if a.config in ("all", "c5") else a.config
    mesh = mg.make_config(name, a.scale)
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
        "config": {"workload": workload_text(name) + "; each step a random sample of %d simplices" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{per_step} random simplices per step of the {ns}-simplex workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------

KERNELS = {3: ["k_prep_vertices", "k_tet_setup<float>", "k_project_tet<float>", "k_project_big<float>",
               "accuracy control (largest cell, second pass, k_project_clip)"],
           2: ["k_prep_vertices", "-", "k_project_warp<2,float>", "-",
               "accuracy control (largest cell, second pass, k_project_clip)"]}


def roofline(dim, st, kern_ms, ns, peaks):
    """The ceiling of the kernel that takes most of the step: issue-bound FP32 arithmetic for the
    projection kernels, from the exact corner incidences of the statistics pass."""
    dom = int(np.argmax(kern_ms[:4]))  # (the accuracy-control slot is several small kernels)
    fp32_peak = peaks.get("fp32_fma_tflops")
    src = "measured (ALU_PEAKS.json, bench_peaks.cu)"
    if fp32_peak is None:
        fp32_peak = 152 * 128 * 2 * 2.070e9 / 1e12
        src = "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (ALU_PEAKS.json absent)"
    if dom == 0:
        hbm = _json_file("MEASURED_PEAKS.json").get("hbm_gbs", 6800.0)
        achieved = st["n_verts"] * (3 * 8 + 8 + 32) / (kern_ms[0] / 1000.0) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": KERNELS[dim][0]}
    if dim == 3 and dom == 3:
        inc = {k: st["large_corners"][i] for i, k in enumerate("abcd")}
    elif dim == 3:
        inc = {k: st["corners_" + k] - st["large_corners"][i] for i, k in enumerate("abcd")}
    else:
        inc = {k: st["corners_" + k] for k in "abcd"}
    flops = sum(FLOPS_PER_INCIDENCE[k] * v for k, v in inc.items())
    sec = kern_ms[dom] / 1000.0
    achieved = flops / sec / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None, "kernel": KERNELS[dim][dom],
            "kernel_ms": kern_ms[dom], "flops_per_launch": flops,
            "flops_per_incidence": FLOPS_PER_INCIDENCE, "peak_source": src,
            "peak_clock_mhz": peaks.get("sm_mhz_median")}
    headline = dim == 3 and dom == 2
    if headline and TRAFFIC_BYTES_PER_TET is not None:
        roof["traffic"] = TRAFFIC_BYTES_PER_TET * ns
        roof["traffic_unit"] = ("bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum of a 1/8 random "
                                "subset of the workload's tetrahedra on its own grid, scaled by tetrahedra")
    if headline and WARP_INST_PER_TET is not None and peaks.get("warp_issue_ginst"):
        inst = WARP_INST_PER_TET * ns / sec / 1e9
        roof["issue"] = {"achieved_ginst": inst, "peak_ginst": peaks["warp_issue_ginst"],
                         "frac": inst / peaks["warp_issue_ginst"],
                         "unit": "warp instructions per second (peak: one per scheduler per clock, measured with "
                                 "FP32 FMAs)"}
    if st.get("n_pieces") and peaks.get("red_f64_run32_gps"):
        red = 2 * st["n_pieces"] / (sum(kern_ms[2:]) / 1000.0) / 1e9
        roof["l2_reductions"] = {"achieved_gps": red, "peak_gps": peaks["red_f64_run32_gps"],
                                 "frac": red / peaks["red_f64_run32_gps"],
                                 "unit": "FP64 reductions per second (two per FP32 piece: the piece and its "
                                         "closure share)"}
    return roof


def _to_dev(torch, dev, mesh):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t(mesh.pos), t(mesh.simplices), t(mesh.rho), torch.empty(mesh.grid, dtype=torch.float64, device=dev)


def bench_projection(a, pkg, proj, dev, stream, name, ws, rank, headline):
    """One workload: FP32-mixed timed, FP64 plain beside it, e2e from pinned host buffers."""
    import torch

    from paper_1509_07720_gb300 import meshgen as mg

    mesh = mg.make_config(name, a.scale)
    ns = mesh.n_simplices
    pos, simp, rho, out = _to_dev(torch, dev, mesh)

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
    st32["n_verts"] = mesh.n_verts

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

    clk = ClockSampler(dev.index)
    clk.start()
    ms32, kern32 = timed(pkg.CDP_FP32_MIXED, a.steps, a.warmup)
    clocks = clk.stop()
    proj.check(stream)
    ms32 = max_over_ranks(ms32, ws, dev)
    value = job_throughput(ws, ns, ms32)
    k64 = max(1, a.fp64_steps)
    ms64, kern64 = timed(pkg.CDP_FP64, k64, 1)
    ms64 = max_over_ranks(ms64, ws, dev)

    e2e = None
    if not a.no_e2e:
        hp = torch.from_numpy(np.ascontiguousarray(mesh.pos)).pin_memory()
        hs = torch.from_numpy(np.ascontiguousarray(mesh.simplices)).pin_memory()
        hr = torch.from_numpy(np.ascontiguousarray(mesh.rho)).pin_memory()
        ho = torch.empty(mesh.grid, dtype=torch.float64).pin_memory()
        dpos, dsimp, drho = torch.empty_like(pos), torch.empty_like(simp), torch.empty_like(rho)

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
        del hp, hs, hr, ho, dpos, dsimp, drho

    amr = None
    lmax = a.amr if a.amr is not None else (3 if name in ("c2", "c4") else 0)
    while lmax > 0 and any(n % (1 << lmax) for n in mesh.grid):
        lmax -= 1
    if lmax > 0:
        # the AMR projection (Sect. 4.4): timed like the exact one, and compared with it: block sums
        # over the coarsest level's cells agree, single cells differ where coarse levels spread mass
        exact = out.clone()
        proj.project(pos, simp, rho, mesh.grid, mesh.box_lo, mesh.box_len, True, precision=pkg.CDP_FP32_MIXED,
                     out=exact, stream=stream)
        _, sta = proj.project_amr(pos, simp, rho, mesh.grid, lmax, mesh.box_lo, mesh.box_len, True,
                                  precision=pkg.CDP_FP32_MIXED, out=out, stream=stream, stats=True)
        b = 1 << lmax
        shp = []
        for n in mesh.grid:
            shp += [n // b, b]
        red = tuple(range(1, 2 * mesh.dim, 2))
        bs_e, bs_a = exact.reshape(shp).sum(dim=red), out.reshape(shp).sum(dim=red)
        scale_e = float(exact.abs().max())
        step_amr = lambda: proj.project_amr(pos, simp, rho, mesh.grid, lmax, mesh.box_lo, mesh.box_len, True,
                                            precision=pkg.CDP_FP32_MIXED, out=out, stream=stream)
        for _ in range(a.warmup):
            step_amr()
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            step_amr()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        msa = max_over_ranks(e0.elapsed_time(e1) / a.steps, ws, dev)
        amr = {"max_level": lmax, "ms_per_step": msa, "value": job_throughput(ws, ns, msa), "unit": UNIT,
               "speedup_vs_exact": ms32 / msa,
               "corners": {k: sta[k] for k in ("corners_a", "corners_b", "corners_c", "corners_d")},
               "block_sum_max_rel_diff": float((bs_e - bs_a).abs().max()) / float(bs_e.abs().max()),
               "cell_max_rel_diff": float((exact - out).abs().max()) / scale_e,
               "what": f"cdp_project_amr, FP32-mixed: every simplex projected exactly onto grid / 2^l, "
                       f"l = min({lmax}, floor(log2 of its smallest height in cells)), then donor-cell gather"}
        del exact, bs_e, bs_a

    peaks = _json_file("ALU_PEAKS.json")
    dim = mesh.dim
    # 3D: vertex records, set-up + main kernel per batch of 2^24, large tetrahedra, then the accuracy
    # control (largest cell, second-pass set-up + main kernel per batch, large tetrahedra, clipping);
    # 2D: vertex records, main kernel, largest cell, second pass, clipping
    batches = max(1, (ns + (1 << 24) - 1) // (1 << 24))
    launches_per_step = 5 if dim == 2 else 1 + 2 * batches + 1 + 1 + 2 * batches + 1 + 1
    line = {
        "metric": METRIC if headline else f"simplices projected/s ({name}), FP32-mixed vs FP64 plain, same GB300",
        "value": value, "unit": UNIT if dim == 3 else "triangles/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-mixed (f64 accumulate)", "data": "synthetic",
        "config": {"workload": workload_text(name, mesh, a.scale), "name": name, "simplices": ns,
                   "grid": list(mesh.grid),
                   "l2": "inputs larger than L2 (no flush)" if ns * 16 > 129e6 else
                         "inputs smaller than L2: steps back to back, warm L2 (no flush)",
                   "parallelism": f"replicas x{ws}"},
        "fp64_plain": {"value": job_throughput(ws, ns, ms64), "unit": UNIT, "ms_per_step": ms64,
                       "kernel_ms": kern64, "speedup_fp32_mixed_vs_fp64": ms64 / ms32},
        "kernel_ms": {k: v for k, v in zip(KERNELS[dim], kern32) if k != "-"},
        "corners": {k: st32[k] for k in ("corners_a", "corners_b", "corners_c", "corners_d", "n_single_cell",
                                         "n_small", "n_large", "n_large_tiles", "n_zero_volume", "exact_fallbacks",
                                         "n_deferred", "n_clipped", "accuracy_bound") if k in st32},
        "roofline": roofline(dim, st32, kern32, ns, peaks),
        "clocks": clocks,
        "gpu_launches": launches_per_step * a.steps,
        "e2e": e2e,
    }
    if amr is not None:
        line["amr"] = amr
    del pos, simp, rho, out
    return line, mesh


def bench_batch(a, pkg, proj, dev, stream, ws, steps=3, warmup=3):
    """The batched workload c5: (1) the 64 projections in one cdp_project_batched call, FP32-mixed and
    FP64; (2) one time step of all 64 problems (drift, vertex density, FP32-mixed projection, FFT
    Poisson, force, kick, drift) replayed as one CUDA graph.  Inputs resident on the device; CUDA
    events around the calls."""
    import torch

    from paper_1509_07720_gb300 import meshgen as mg

    batch = mg.make_batch("c5")
    dt = mg.cfl_dt(batch)
    keep = []
    probs = []
    flat = []
    for p in batch:
        m = p.mesh
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        pos = [t(m.pos[a_]) for a_ in range(m.dim)]
        vel = [t(p.vel[a_]) for a_ in range(m.dim)]
        acc = [torch.zeros(m.n_verts, dtype=torch.float64, device=dev) for _ in range(m.dim)]
        simp, mass = t(m.simplices), t(p.masses)
        rho = torch.zeros(m.n_verts, dtype=torch.float64, device=dev)
        rho0 = t(m.rho)
        cm = torch.zeros(m.grid, dtype=torch.float64, device=dev)
        cm2 = torch.zeros(m.grid, dtype=torch.float64, device=dev)
        phi = torch.zeros(m.grid, dtype=torch.float64, device=dev)
        sp = pkg.cdp_step_problem()
        sp.mesh = pkg.Projector.make_problem(pos, simp, rho, m.grid, m.box_lo, m.box_len, True, cm)
        for a_ in range(m.dim):
            sp.vel[a_] = vel[a_].data_ptr()
            sp.acc[a_] = acc[a_].data_ptr()
        sp.simplex_mass = mass.data_ptr()
        sp.phi = phi.data_ptr()
        probs.append(sp)
        flat.append(pkg.Projector.make_problem(pos, simp, rho0, m.grid, m.box_lo, m.box_len, True, cm2))
        keep.append((pos, vel, acc, simp, mass, rho, rho0, cm, cm2, phi))
    ns = sum(p.mesh.n_simplices for p in batch)
    st = stream.cuda_stream

    def time_calls(fn, n_steps, n_warm):
        for _ in range(n_warm):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n_steps

    def project_all(prec):
        rc = pkg.cdp_project_batched(proj._ctx, flat, prec, st)
        if rc:
            raise RuntimeError(f"cdp_project_batched: {rc}")

    clk = ClockSampler(dev.index)
    clk.start()
    ms_p32 = time_calls(lambda: project_all(pkg.CDP_FP32_MIXED), steps, warmup)
    clocks = clk.stop()
    ms_p64 = time_calls(lambda: project_all(pkg.CDP_FP64), 1, 1)
    arr = (pkg.cdp_step_problem * len(probs))(*probs)

    def step():
        rc = pkg.cdp_step_batched(proj._ctx, arr, pkg.CDP_FP32_MIXED, dt, 1.0, True, st)
        if rc:
            raise RuntimeError(f"cdp_step_batched: {rc}")

    ms_step = time_calls(step, steps, warmup)  # the first warm-up call captures the graph
    proj.check(stream)
    ms_p32 = max_over_ranks(ms_p32, ws, dev)
    ms_step = max_over_ranks(ms_step, ws, dev)
    del keep
    return {"workload": workload_text("c5"), "problems": len(batch), "simplices": ns,
            "projection": {"ms_per_step": ms_p32, "simplices_per_s": job_throughput(ws, ns, ms_p32),
                           "fp64_ms_per_step": ms_p64, "fp64_simplices_per_s": job_throughput(ws, ns, ms_p64),
                           "speedup_fp32_mixed_vs_fp64": ms_p64 / ms_p32},
            "step": {"ms_per_step": ms_step, "simplices_per_s": job_throughput(ws, ns, ms_step),
                     "what": "drift, vertex density, FP32-mixed projection, FFT Poisson, force, kick, drift; "
                             "one CUDA graph"},
            "dtype": "f32-mixed projection, f64 solver", "steps": steps, "warmup": warmup, "clocks": clocks}


def run_ours(a):
    import torch

    import paper_1509_07720_gb300 as pkg
    from paper_1509_07720_gb300 import build

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    build.build_library()
    proj = pkg.Projector(local)
    stream = torch.cuda.current_stream(dev)
    names = ["c3", "c1a", "c1b", "c2", "c4", "c5"] if a.config == "all" else [a.config]
    for name in names:
        if name == "c5":
            b = bench_batch(a, pkg, proj, dev, stream, ws, steps=max(3, min(a.steps, 10)), warmup=max(3, a.warmup))
            if rank == 0:
                line = {"metric": "simplices projected/s, 64 independent problems (c5), FP32-mixed, same GB300",
                        "value": b["projection"]["simplices_per_s"], "unit": "simplices/s", "n_gpus": ws,
                        "steps": b["steps"], "warmup": b["warmup"], "ms_per_step": b["projection"]["ms_per_step"],
                        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                        "dtype": "f32-mixed (f64 accumulate)", "data": "synthetic",
                        "config": {"workload": b["workload"], "name": "c5", "simplices": b["simplices"],
                                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"},
                        "batched": b, "clocks": b["clocks"], "e2e": None}
                print(json.dumps(line), flush=True)
            continue
        headline = name == WORKLOAD
        line, mesh = bench_projection(a, pkg, proj, dev, stream, name, ws, rank, headline)
        if headline and a.config != "all" and not a.no_batched:
            line["batched"] = bench_batch(a, pkg, proj, dev, stream, ws)
        if rank == 0:
            if headline and ws == 1 and not a.no_cpu_baseline:
                line["cpu_baseline"] = _cpu_baseline(mesh)
            print(json.dumps(line), flush=True)
        del mesh
    proj.close()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
