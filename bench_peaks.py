#!/usr/bin/env python
"""Measured ceilings for the roofline of the projection kernels (micro-benchmarks, one GPU).

The projection is not a dense contraction and moves little memory, so its ceilings are arithmetic
issue rates and L2 reduction throughput, which MEASURED_PEAKS.json (HBM copy, bf16 GEMM) does not
cover.  This script compiles ``bench_peaks.cu`` (in-tree ``bench_peaks.so``), runs each kernel a
few times with CUDA events while ``nvidia-smi`` samples the SM clock, and writes ``ALU_PEAKS.json``:

  fp32_fma_tflops    FP32 FMA throughput (2 flops per FMA), all SMs, 8 independent chains/thread
  fp64_fma_tflops    FP64 FMA throughput
  int32_alu_tops     INT32 add + xor throughput (2 ops per step)
  int32_imad_tops    INT32 multiply-add throughput (2 ops)
  red_f64_rand_gps   scattered FP64 reductions into a 256^3 FP64 grid, every lane a random cell
  red_f64_run32_gps  the same with a warp covering 32 consecutive cells (one box row of the flush)
  warp_issue_ginst   FP32 FMA warp instructions per second (a lower bound of the issue peak)
and the median SM clock under load, so each figure can be rescaled to another clock.

Usage: python bench_peaks.py [--out ALU_PEAKS.json]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(ROOT, "bench_peaks.cu")
LIB = os.path.join(ROOT, "bench_peaks.so")
JSON_PATH = os.path.join(ROOT, "ALU_PEAKS.json")


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
                               "-Xcompiler", "-fPIC", "-shared", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def load():
    lib = ctypes.CDLL(build())
    lib.peaks_alu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.peaks_alu.restype = ctypes.c_float
    lib.peaks_red_f64.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.peaks_red_f64.restype = ctypes.c_float
    lib.peaks_device_sms.argtypes = []
    lib.peaks_device_sms.restype = ctypes.c_int
    return lib


def _clock_sampler(dev):
    try:
        return subprocess.Popen(["nvidia-smi", "-i", str(dev), "--query-gpu=clocks.sm,clocks.max.sm,power.draw",
                                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                                stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_stop(p):
    if p is None:
        return None, None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
        out, _ = p.communicate()
    sm, smax = [], []
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        try:
            sm.append(float(f[0]))
            smax.append(float(f[1]))
        except (ValueError, IndexError):
            continue
    return (statistics.median(sm) if sm else None), (max(smax) if smax else None)


def measure(device: int = 0) -> dict:
    """Run every micro-benchmark on the current CUDA device and return the figures."""
    lib = load()
    sms = lib.peaks_device_sms()
    if sms <= 0:
        raise RuntimeError("no CUDA device")
    blocks = sms * 8  # 2048 threads per SM
    res = {"sms": sms, "blocks": blocks, "threads_per_block": 256}
    ops = ctypes.c_double(0.0)
    clk = _clock_sampler(device)
    time.sleep(0.2)
    # (kind, iterations per thread, repetitions): each launch takes about 10-50 ms
    for key, kind, iters, reps in (("fp32_fma_tflops", 0, 20000, 10), ("fp64_fma_tflops", 1, 300, 5),
                                   ("int32_alu_tops", 2, 20000, 10), ("int32_imad_tops", 3, 20000, 10)):
        ms = lib.peaks_alu(kind, blocks, iters, reps, ctypes.byref(ops))
        if ms <= 0:
            raise RuntimeError(f"{key}: CUDA error")
        res[key] = ops.value / (ms * 1e-3) / 1e12
        res[key.replace("_tflops", "_ms").replace("_tops", "_ms")] = ms
    # FP32 FMA warp instructions per second: 32 lanes x 2 flops per warp instruction
    res["warp_issue_ginst"] = res["fp32_fma_tflops"] * 1e12 / 64.0 / 1e9
    n = 256 ** 3
    per = 1024
    for key, run in (("red_f64_rand_gps", 1), ("red_f64_run32_gps", 32)):
        ms = lib.peaks_red_f64(n, blocks, per, run, 5)
        if ms <= 0:
            raise RuntimeError(f"{key}: CUDA error")
        res[key] = blocks * 256 * per / (ms * 1e-3) / 1e9
    res["red_grid_cells"] = n
    sm, smax = _clock_stop(clk)
    res["sm_mhz_median"] = sm
    res["sm_max_mhz"] = smax
    return res


def read_json(path: str = JSON_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=JSON_PATH)
    a = ap.parse_args(argv)
    import torch  # noqa: F401  (the CUDA context of the device the bench uses)

    res = measure(0)
    try:
        name = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=name", "--format=csv,noheader"],
                              capture_output=True, text=True).stdout.strip()
    except OSError:
        name = None
    res["gpu_name"] = name
    res["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    res["how"] = ("bench_peaks.cu kernels timed with CUDA events (mean of 5-10 launches after one warm-up), "
                  "8 blocks of 256 threads per SM; nvidia-smi clock samples every 100 ms during the runs")
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    sys.exit(main())
