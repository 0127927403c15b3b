"""Named projection cases for profiling (ncu) and timing: ``python profile_cases.py <case>``.

Measurement harness beside ``bench.py``, not part of the library: each case builds its seeded
synthetic mesh, puts it on ``cuda:0`` and projects it ``--reps`` times through the public API
(``Projector.project``) with CUDA events around every call, then prints one JSON line with the
times.  ``--amr L`` projects through the levels 0 .. L with donor-cell gather
(``Projector.project_amr``) instead of the exact projection.  Cases:

  c3           the 128^3 Kuhn lattice of the headline benchmark (``--scale n``: an n^3 lattice;
               ``--subset k``: a seeded random 1/k of its tetrahedra on the same grid, the size an
               ncu capture of the full kernel allows)
  c4           the bisected adaptive mesh (simplex volumes over four decades; ``--scale n``: an n^3
               base lattice, default 64, grid 8n)
  c5           one problem of the 64-problem batched workload (``--problem i``), projected alone
  c5_3d        the 32 three-dimensional problems of that workload, one after the other
  c5_batch     all 64 problems in one cdp_project_batched call (one launch of each kernel per group
               of problems of one dimension)
  c5_2d        the 32 two-dimensional problems of that workload in one cdp_project_batched call
  c5_step      one time step of all 64 problems (cdp_step_batched: drift, vertex density, projection,
               FFT Poisson, force, kick, drift), enqueued eagerly (no graph) so that every launch shows
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def _device_mesh(torch, mesh):
    d = torch.device("cuda:0")
    return (torch.from_numpy(np.ascontiguousarray(mesh.pos)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.simplices)).to(d),
            torch.from_numpy(np.ascontiguousarray(mesh.rho)).to(d),
            torch.empty(tuple(mesh.grid), dtype=torch.float64, device=d))


def _step_case(a, torch, pkg, mg, proj, stream, prec):
    """One time step of the 64 problems, eagerly enqueued, timed with CUDA events per repetition."""
    d = torch.device("cuda:0")
    batch = mg.make_batch("c5")
    dt = mg.cfl_dt(batch)
    keep, probs = [], []
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(d)
    for p in batch:
        m = p.mesh
        pos = [t(m.pos[k]) for k in range(m.dim)]
        vel = [t(p.vel[k]) for k in range(m.dim)]
        acc = [torch.zeros(m.n_verts, dtype=torch.float64, device=d) for _ in range(m.dim)]
        simp, mass = t(m.simplices), t(p.masses)
        rho = torch.zeros(m.n_verts, dtype=torch.float64, device=d)
        cm = torch.zeros(m.grid, dtype=torch.float64, device=d)
        phi = torch.zeros(m.grid, dtype=torch.float64, device=d)
        sp = pkg.cdp_step_problem()
        sp.mesh = pkg.Projector.make_problem(pos, simp, rho, m.grid, m.box_lo, m.box_len, True, cm)
        for k in range(m.dim):
            sp.vel[k] = vel[k].data_ptr()
            sp.acc[k] = acc[k].data_ptr()
        sp.simplex_mass = mass.data_ptr()
        sp.phi = phi.data_ptr()
        probs.append(sp)
        keep.append((pos, vel, acc, simp, mass, rho, cm, phi))
    arr = (pkg.cdp_step_problem * len(probs))(*probs)
    times = []
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = pkg.cdp_step_batched(proj._ctx, arr, prec, dt, 1.0, False, stream.cuda_stream)
        if rc:
            raise SystemExit(f"cdp_step_batched: {rc}")
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    proj.check(stream)
    print(json.dumps({"case": "c5_step", "prec": a.prec, "simplices": int(sum(p.mesh.n_simplices for p in batch)),
                      "ms_per_rep": times}), flush=True)
    proj.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["c3", "c4", "c5", "c5_3d", "c5_batch", "c5_2d", "c5_step"])
    ap.add_argument("--scale", type=int, default=None, help="c3: lattice size (default 128)")
    ap.add_argument("--subset", type=int, default=1, help="c3: keep a random 1/k of the tetrahedra (seed 8)")
    ap.add_argument("--problem", type=int, default=0, help="c5: problem index in [0, 64)")
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--stats", action="store_true", help="also one instrumented pass and per-kernel times")
    ap.add_argument("--accuracy-off", action="store_true", help="no accuracy control")
    ap.add_argument("--amr", type=int, default=None, help="project through the levels 0 .. AMR (grid / 2^level)")
    a = ap.parse_args(argv)

    import os
    import sys

    import torch

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import paper_1509_07720_gb300 as pkg
    from paper_1509_07720_gb300 import build
    from paper_1509_07720_gb300 import meshgen as mg

    if not torch.cuda.is_available():
        raise SystemExit("profile_cases needs a CUDA device")
    build.build_library()
    if a.case in ("c3", "c4"):
        m = mg.make_config(a.case, a.scale)
        if a.subset > 1:
            rng = np.random.default_rng(8)
            m = m.subset(np.sort(rng.choice(m.n_simplices, m.n_simplices // a.subset, replace=False)))
        meshes = [m]
    else:
        batch = mg.make_batch("c5")
        if a.case == "c5":
            meshes = [batch[a.problem].mesh]
        elif a.case == "c5_3d":
            meshes = [p.mesh for p in batch if p.mesh.dim == 3]
        elif a.case == "c5_batch":
            meshes = [p.mesh for p in batch]
        elif a.case == "c5_2d":
            meshes = [p.mesh for p in batch if p.mesh.dim == 2]
        else:
            meshes = []  # (c5_step builds its own problems)
    data = [(m, *_device_mesh(torch, m)) for m in meshes]
    prec = pkg.CDP_FP32_MIXED if a.prec == "fp32" else pkg.CDP_FP64
    if a.accuracy_off:
        prec |= pkg.CDP_ACCURACY_OFF
    proj = pkg.Projector(0)
    stream = torch.cuda.current_stream()
    if a.case == "c5_step":
        return _step_case(a, torch, pkg, mg, proj, stream, prec)
    times = []
    probs = [pkg.Projector.make_problem(pos, simp, rho, m.grid, m.box_lo, m.box_len, m.periodic, out)
             for m, pos, simp, rho, out in data]
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if a.case in ("c5_batch", "c5_2d"):
            rc = pkg.cdp_project_batched(proj._ctx, probs, prec, stream.cuda_stream)
            if rc:
                raise SystemExit(f"cdp_project_batched: {rc}")
        elif a.amr is not None:
            for m, pos, simp, rho, out in data:
                proj.project_amr(pos, simp, rho, m.grid, a.amr, m.box_lo, m.box_len, m.periodic, precision=prec,
                                 out=out, stream=stream)
        else:
            for m, pos, simp, rho, out in data:
                proj.project(pos, simp, rho, m.grid, m.box_lo, m.box_len, m.periodic, precision=prec, out=out,
                             stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    proj.check(stream)
    extra = {}
    if a.stats:
        proj.timing(True)
        for m, pos, simp, rho, out in data:
            if a.amr is not None:
                proj.project_amr(pos, simp, rho, m.grid, a.amr, m.box_lo, m.box_len, m.periodic, precision=prec,
                                 out=out, stream=stream)
            else:
                proj.project(pos, simp, rho, m.grid, m.box_lo, m.box_len, m.periodic, precision=prec, out=out,
                             stream=stream)
        kern, calls = proj.timing()
        proj.timing(False)
        extra["kernel_ms"] = dict(zip(["vertex records", "set-up", "main", "large", "accuracy control"], kern))
        if a.amr is not None:
            extra["stats"] = [proj.project_amr(pos, simp, rho, m.grid, a.amr, m.box_lo, m.box_len, m.periodic,
                                               precision=prec, out=out, stream=stream, stats=True)[1]
                              for m, pos, simp, rho, out in data]
        else:
            extra["stats"] = [proj.project(pos, simp, rho, m.grid, m.box_lo, m.box_len, m.periodic, precision=prec,
                                           out=out, stream=stream, stats=True)[1] for m, pos, simp, rho, out in data]
    print(json.dumps({**extra, "case": a.case, "scale": a.scale, "subset": a.subset, "problem": a.problem if a.case == "c5" else None,
                      "prec": a.prec, "simplices": int(sum(m.n_simplices for m in meshes)),
                      "amr": a.amr, "ms_per_rep": times}), flush=True)
    proj.close()


if __name__ == "__main__":
    main()
