"""Benchmark of the AIM operator products on GB300.

Workload (default): the lossy-conductor sphere -- radius 1 mm, sigma = 5.8e7 S/m,
10 GHz, icosphere of 20,480 triangles (30,720 RWG edges), exterior AIM grid
64^3 physical (128^3 FFT), complex128, stencil order 2, near radius 5, one
right-hand side; the interior operator is near-region only (5 skin depths fit
in the near region).  Inputs are seeded and synthetic.

One step applies the exterior L0 and K0 AIM products and the interior LI and
KI near-region products to one vector (the operator work of one system
matvec).  value = RWG unknowns x steps / s, whole job.

--impl reference times the CPU oracle (numpy FFT grid products) on the same
workload and metric.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RWG-unknown matvecs/s"
UNIT = "RWG-unknown matvecs/s"
L2_BYTES = 129 * 2 ** 20


def workload(name):
    from synth import icosphere
    if name == "lossy-sphere-30720":
        V, T = icosphere(5, 1e-3)
        return dict(V=V, T=T, f=10e9, eps_r=1.0, sigma=5.8e7, grid_n=64,
                    desc="copper sphere r=1mm, sigma=5.8e7 S/m, 10 GHz, 20480 triangles / 30720 RWG, "
                         "grid 64^3 (FFT 128^3), complex128, near-only interior, 1 RHS")
    if name == "dielectric-sphere-1920":
        V, T = icosphere(3, 1e-2)
        return dict(V=V, T=T, f=3e9, eps_r=4.0, sigma=0.0, grid_n=0,
                    desc="dielectric sphere r=1cm, eps_r=4, 3 GHz, 1280 triangles / 1920 RWG, h=0.5 mean edge, "
                         "complex128, AIM interior, 1 RHS")
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, gpu):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
            "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
            "clocks_event_reasons.sw_power_cap"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def stage_model(stage, info, ne, nt, nnz_ext, nnz_int):
    """Algorithmic bytes and FLOPs of ONE launch of a stage (FP64 complex = 16 B)."""
    N = info[0:3].astype(np.int64)
    n = info[3:6].astype(np.int64)
    Nx, Ny, Nz = N
    nx, ny, nz = n
    c = 16
    fl = lambda length, pencils: 5.0 * length * np.log2(length) * pencils
    table = {
        "fft_fwd_x": ((Nx * Ny * Nz + nx * Ny * Nz) * c, fl(nx, Ny * Nz)),
        "fft_fwd_y": ((nx * Ny * Nz + nx * ny * Nz) * c, fl(ny, nx * Nz)),
        "fft_fwd_z": ((nx * ny * Nz + nx * ny * nz) * c, fl(nz, nx * ny)),
        "fft_inv_z": ((nx * ny * nz + nx * ny * Nz) * c, fl(nz, nx * ny)),
        "fft_inv_y": ((nx * ny * Nz + nx * Ny * Nz) * c, fl(ny, nx * Nz)),
        "fft_inv_x": ((nx * Ny * Nz + Nx * Ny * Nz) * c, fl(nx, Ny * Nz)),
        "spmv_aim": (nnz_ext * (c + 4) + (ne + 1) * 8 + 3 * ne * c, 8.0 * nnz_ext),
        "spmv_near_only": (nnz_int * (c + 4) + (ne + 1) * 8 + 3 * ne * c, 8.0 * nnz_int),
    }
    return table.get(stage)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2003_11679_gb300 as sie
    from paper_2003_11679_gb300 import build as libbuild
    from synth import cn_vector

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    libbuild.build()
    wl = workload(args.workload)
    stream = torch.cuda.Stream()
    ctx = sie.Context(local, stream=stream.cuda_stream)
    mesh = sie.Mesh(ctx, wl["V"], wl["T"])
    t0 = time.time()
    op = sie.Operator(mesh, wl["f"], wl["eps_r"], 1.0, wl["sigma"], sie.params(grid_n=wl["grid_n"]))
    build_s = time.time() - t0
    info = op.info()
    ne, nt = mesh.ne, mesh.nt
    nnz_int = op.near_csr(2)[0][-1]
    x = torch.from_numpy(cn_vector(ne, 1 + rank)).to(f"cuda:{local}")
    ys = [torch.zeros_like(x) for _ in range(4)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")

    def step():
        for w in range(4):
            op.matvec(w, x, ys[w])

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ctx.profile(True)
        with Clocks(local) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))  # L2 flush between timed steps (outside the events)
                starts[i].record(stream)
                step()
                ends[i].record(stream)
            torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        # end to end through host buffers (H2D of x and D2H of y inside)
        xh = cn_vector(ne, 1 + rank)
        yh = np.zeros_like(xh)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for i in range(args.steps):
            for w in range(4):
                op.matvec(w, xh, yh)
        e2e_s = time.perf_counter() - t1
    if world > 1:
        t = torch.tensor([ms, e2e_s], device=f"cuda:{local}", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e_s = float(t[0]), float(t[1])
    if rank != 0:
        return
    value = world * ne * args.steps / (ms * 1e-3)
    peaks, kind = measured_peaks()
    # dominant stage and its roofline
    dom = max(prof, key=lambda k: prof[k][0])
    dms, dcount = prof[dom]
    model = stage_model(dom, info, ne, nt, info[8], nnz_int)
    roof = None
    if model is not None:
        B, F = model
        avg_s = dms * 1e-3 / dcount
        roof = {"bound": "hbm", "kernel": dom, "achieved": B / avg_s / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": B / avg_s / 1e9 / peaks["hbm_gbs"], "traffic": None,
                "flops_per_launch": F, "fp64_tflops_achieved": F / avg_s / 1e12, "peak_kind": kind,
                "avg_launch_us": avg_s * 1e6, "launches": dcount}
    launches = sum(c for _, c in prof.values())
    cpu = cpu_baseline(wl, args) if not args.no_cpu else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "ne": ne, "nt": nt,
                   "grid_N": info[0:3].tolist(), "fft_n": info[3:6].tolist(), "near_nnz_ext": int(info[8]),
                   "near_nnz_int": int(nnz_int), "step": "L0+K0 (exterior AIM) + LI+KI (interior near) products",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "build_s": build_s},
        "e2e": {"value": world * ne * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * ne * 16,
                "d2h_bytes_per_step": 4 * ne * 16},
        "gpu_launches": launches,
        "stages_ms": {k: round(v[0], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "roofline": roof,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))


def cpu_baseline(wl, args):
    """The oracle's FP64 AIM grid products on the host cores (bounded sample)."""
    from oracle import aim
    from oracle.rwg import Mesh
    from synth import cn_vector
    m = Mesh(wl["V"], wl["T"])
    g = aim.grid_params(m, M=2, grid_n=wl["grid_n"] or None)
    k0 = 2 * np.pi * wl["f"] / 299792458.0
    A = aim.AIM(m, k0, g, near=False)
    x = cn_vector(m.ne, 1)
    reps = 0
    t0 = time.perf_counter()
    while True:
        A.grid_L(x)
        A.grid_K(x)
        reps += 1
        if time.perf_counter() - t0 > args.cpu_seconds or reps >= 50:
            break
    dt = (time.perf_counter() - t0) / reps
    return {"value": m.ne / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"exterior grid products L0+K0 only (7 numpy FFT convolutions at the full grid), {reps} reps; "
                      "near-region products excluded, so the CPU time per step is understated"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args.workload)
    t0 = time.perf_counter()
    cpu = cpu_baseline(wl, args)
    line = {"metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * (1.5 * len(wl["T"])) / cpu["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": {"kind": cpu["kind"], "cores": cpu["cores"], "sample": cpu["sample"],
                             "value": cpu["value"]},
            "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lossy-sphere-30720")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
