"""Benchmark of the AIM operator products on GB300.

Workload (default): the lossy-conductor sphere -- radius 1 mm, sigma = 5.8e7 S/m,
10 GHz, icosphere of 20,480 triangles (30,720 RWG edges), exterior AIM grid
64^3 physical (128^3 FFT), complex128, stencil order 2, near radius 5, one
right-hand side; the interior operator is near-region only (5 skin depths fit
in the near region).  Inputs are seeded and synthetic.

One step is one product with the GIBC system matrix of Eq. (sys) (AEFIE form,
unknowns [H; c0 rho]): the interior impedance Z_i H by the nested near-region
solve, seven source grids projected, 7 forward + 4 inverse pruned 3D FFTs,
spectral multiply with G and grad G, interpolation, and the precorrected
near-region products.  value = RWG unknowns x system matvecs / s, whole job.
The JSON line also reports GMRES solves/s and p50/p99 solve latency of the
dielectric-sphere workload (1,920 RWG, equal-volume mesh), FP64 and with
mixed-precision iterative refinement on the same right-hand sides, each solve's
backscatter RCS checked against the Mie series (1%).

A ports leg drives a copper bar through two delta-gap ports (sie_port_*) and
reports its admittance and S parameters at a few frequencies, with the
near-region-only interior and with the surface impedance comparator.

The FP64 path's roofline fractions use the FP64 FMA throughput the library's
probe kernel measures in the same run (sie_probe_fma).

--impl reference (and the cpu_baseline object) time the oracle's system
product of Eq. (sys) -- AIM exterior with its near terms, near-region-only
interior Z' by a sparse LU -- on a bounded sample of the workload: the same
sphere, material and exterior grid (the same 128^3 FFT convolutions) on a
320-triangle mesh.  The grid part dominates its cost and has the full size, so
N_e(full) / (step time) is an upper bound of the oracle's full-size throughput.
"""
import argparse
import json
import os
import platform
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


LOSSY_LEVELS = {"lossy-sphere-30720": 5, "lossy-sphere-7680": 4, "lossy-sphere-1920": 3, "lossy-sphere-480": 2}


def workload(name):
    from synth import icosphere
    if name in LOSSY_LEVELS:
        lev = LOSSY_LEVELS[name]
        V, T = icosphere(lev, 1e-3)
        nt = 20 * 4 ** lev
        return dict(V=V, T=T, f=10e9, eps_r=1.0, sigma=5.8e7, grid_n=64, radius=1e-3, level=lev,
                    desc=f"copper sphere r=1mm, sigma=5.8e7 S/m, 10 GHz, {nt} triangles / {3 * nt // 2} RWG, "
                         "grid 63^3 (grid_n 64, FFT 128^3), complex128, near-only interior, 1 RHS")
    if name == "dielectric-sphere-1920":
        V, T = icosphere(3, 1e-2, equal_volume=True)
        return dict(V=V, T=T, f=3e9, eps_r=4.0, sigma=0.0, grid_n=0, radius=1e-2, level=3,
                    desc="dielectric sphere r=1cm, eps_r=4, 3 GHz, 1280 triangles / 1920 RWG (equal-volume "
                         "icosphere), h=0.5 mean edge, complex128, AIM interior, 1 RHS")
    raise SystemExit(f"unknown workload {name}")


def mie_backscatter(name):
    """The Mie-series backscatter RCS of a workload's sphere, as stored by
    tests/golden/make_mie_backscatter.py (from the oracle's Mie series)."""
    if name in LOSSY_LEVELS:
        name = "lossy-sphere-30720"  # the same sphere at every mesh level
    path = os.path.join(ROOT, "tests", "golden", "mie_backscatter.txt")
    for line in open(path):
        f = line.split()
        if f and f[0] == name:
            return float(f[5])
    raise KeyError(name)


def cpu_info():
    """Host CPU model (lscpu, else platform) and logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return model or platform.processor() or platform.machine(), os.cpu_count()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(ms, e2e_s, world, device):
    """Whole-job times of a replicas run: the slowest rank sets them (max over
    ranks of the timed-region milliseconds and of the end-to-end seconds)."""
    if world == 1:
        return ms, e2e_s
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, e2e_s], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0]), float(t[1])


def job_value(world, ne, steps, ms):
    """RWG unknowns x system matvecs per second over all ranks (each rank runs
    its own replica of the workload)."""
    return world * ne * steps / (ms * 1e-3)


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
    """Algorithmic bytes and FLOPs of ONE launch of a stage (FP64 complex = 16 B).
    FFT passes: one read of the pencils' live input and one write of the
    output, 5 n log2 n flops per pencil (radix-2 operation count), times the
    grids one launch transforms (FFT_GRIDS)."""
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
        "spai_apply": (nnz_int * (c + 4) + (ne + 1) * 8 + 3 * ne * c, 8.0 * nnz_int),
        "specmul_sys": ((7 + 4 + 4) * nx * ny * nz * c, 8 * 10.0 * nx * ny * nz),
        # fused forward z (7 grids) + spectral products + inverse z (4 grids):
        # the z < Nz planes in and out, the 4 kernel spectra in
        "fft_z_specmul": ((11 * nx * ny * Nz + 4 * nx * ny * nz) * c,
                          11 * fl(nz, nx * ny) + 8 * 10.0 * nx * ny * nz),
        # two edge CSR products sharing the pattern (LA H and K E: 2 values + 1 col per nnz),
        # Ix E (5 nnz/row), triangle Lphi product (info[7] pairs), vectors
        "spmv_sys": (nnz_ext * (2 * c + 4) + 5 * ne * (c + 4) + int(info[7]) * (c + 4) + 8 * ne * c + 6 * nt * c,
                     16.0 * nnz_ext + 8.0 * int(info[7])),
        # k_spmv2 alone: both value arrays and the columns once, row pointers,
        # H and E read once, y read and written
        "spmv_near_ext": (nnz_ext * (2 * c + 4) + (ne + 1) * 8 + 4 * ne * c, 16.0 * nnz_ext),
        # the rest of the product's sparse steps: I-cross E, triangle Lphi, vectors
        "spmv_sys_rest": (5 * ne * (c + 4) + int(info[7]) * (c + 4) + 4 * ne * c + 6 * nt * c, 8.0 * int(info[7])),
    }
    r = table.get(stage)
    if r is not None and stage in FFT_GRIDS:
        r = (r[0] * FFT_GRIDS[stage], r[1] * FFT_GRIDS[stage])
    return r


# grids per FFT launch in the system product: 7 forward (H, E, rho sources), 4 inverse
FFT_GRIDS = {"fft_fwd_x": 7, "fft_fwd_y": 7, "fft_fwd_z": 7, "fft_inv_z": 4, "fft_inv_y": 4, "fft_inv_x": 4}

# DRAM bytes (read + write) per launch of a stage's kernels from one ncu capture
# (profiles/), keyed by stage and path, with the hash of the library sources
# the capture was taken at: a stale entry (kernels changed since) reads as null.
# DRAM bytes (read + write) per launch of a stage's kernel from one ncu capture,
# with the hash of the library sources it was taken on (stale once they change).
# k_fft_z_sys<7,2,double2> on the 128^3 FFT grid: the grid part has the same
# size at every mesh level of the copper workload, so the capture on the
# 480-RWG mesh holds per launch for the 30,720-RWG one.
TRAFFIC = {("fft_z_specmul", "fp64"): (249870080 + 47390208, "f124e1ac95d297f3")}


def source_hash():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2003_11679_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_of(stage, path):
    e = TRAFFIC.get((stage, path))
    return e[0] if e and e[1] == source_hash() else None



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
    fp64_peak, fp32_peak = sie.probe_fma(local)  # FMA throughput, measured here
    stream = torch.cuda.Stream()
    ctx = sie.Context(local, stream=stream.cuda_stream)
    mesh = sie.Mesh(ctx, wl["V"], wl["T"])
    t0 = time.time()
    model = sie.SIE_SIBC if args.interior == "sibc" else sie.SIE_GIBC
    op = sie.Operator(mesh, wl["f"], wl["eps_r"], 1.0, wl["sigma"],
                      sie.params(grid_n=wl["grid_n"], interior_model=model))
    build_s = time.time() - t0
    info = op.info()
    ne, nt = mesh.ne, mesh.nt
    nnz_int = op.near_csr(2)[0][-1] if args.interior == "gibc" else 0
    n = ne + nt
    x = torch.from_numpy(cn_vector(n, 1 + rank)).to(f"cuda:{local}")
    y = torch.zeros_like(x)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")

    def step():
        op.matvec(sie.SIE_OP_SYS, x, y)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

        def timed(profile, label="timed"):
            """K steps, L2 flushed between them (outside the events); with
            profile=True the library's per-stage CUDA events are recorded too.
            The unprofiled loop sits in an NVTX range named `label` (for ncu
            --nvtx-include)."""
            ctx.profile(profile)
            if not profile:
                torch.cuda.nvtx.range_push(label)
            for i in range(args.steps):
                flush.fill_(float(i))
                starts[i].record(stream)
                step()
                ends[i].record(stream)
            torch.cuda.synchronize()
            if not profile:
                torch.cuda.nvtx.range_pop()
            pr = ctx.profile_read() if profile else None
            ctx.profile(False)
            return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), pr

        with Clocks(local) as clk:
            ms, _ = timed(False, "sie_fp64")  # the reported step time: no stage events
            if world > 1:
                dist.barrier()
            ginfo, gstats = op.info(), op.stats()  # graph nodes and nested iterations of the timed loop
            ms_prof, prof = timed(True)     # stage breakdown and roofline kernel times
        nested = op.stats()
        graph_state = int(ginfo[16])  # +1: FP64 system-product graph captured (used by the timed loop)
        # end to end through host buffers (H2D of x and D2H of y inside the call)
        xh = cn_vector(n, 1 + rank)
        yh = np.zeros_like(xh)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for i in range(args.steps):
            op.matvec(sie.SIE_OP_SYS, xh, yh)
        e2e_s = time.perf_counter() - t1
        # complex64 grid path (SIE_MIXED) on the same workload
        op.set_solver(precision=sie.SIE_MIXED)
        y64 = y.clone()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ms32, _ = timed(False, "sie_mixed")
        _, prof32 = timed(True)
        op.set_solver(precision=sie.SIE_FP64)
        op.matvec(sie.SIE_OP_SYS, x, y64)
        op.set_solver(precision=sie.SIE_MIXED)
        op.matvec(sie.SIE_OP_SYS, x, y)
        op.set_solver(precision=sie.SIE_FP64)
        torch.cuda.synchronize()
        # current rows (the grid product lives there; the charge rows are exact in both)
        mixed_err = float((y[:ne] - y64[:ne]).abs().norm() / y64[:ne].abs().norm())
        block = block_stats(sie, op, ne, stream, args)
    solves = solve_stats(sie, ctx, args) if not args.no_solve else None
    lossy_solves = lossy_solve_stats(sie, op, args, wl) if not args.no_solve else None
    batching = None
    if not args.no_solve and args.batch_rhs > 0 and rank == 0:
        try:
            batching = batching_stats(sie, ctx, args)
        except Exception as e:  # reported, not fatal to the line
            batching = {"error": f"{type(e).__name__}: {e}"[:300]}
    ports = None
    if not args.no_solve and args.port_freqs and rank == 0:
        try:
            ports = ports_stats(sie, ctx, args)
        except Exception as e:  # reported, not fatal to the line
            ports = {"error": f"{type(e).__name__}: {e}"[:300]}
    serving = None
    if not args.no_solve and args.serve_requests > 0 and rank == 0:
        try:
            serving = serving_stats(args)
        except Exception as e:  # the trace's failure is reported, not fatal to the line
            serving = {"error": f"{type(e).__name__}: {e}"[:300]}
    ms, e2e_s = combine_ranks(ms, e2e_s, world, f"cuda:{local}")
    if rank != 0:
        return
    value = job_value(world, ne, args.steps, ms)
    peaks, kind = measured_peaks()
    # dominant kernel stage (solver bookkeeping stages excluded) and its roofline
    kern = {k: v for k, v in prof.items() if k not in ("inner_solve", "constraint_solve")}
    dom = max(kern, key=lambda k: kern[k][0])
    dms, dcount = kern[dom]
    model = stage_model(dom, info, ne, nt, info[8], nnz_int)
    roof = None
    if model is not None:
        B, F = model
        avg_s = dms * 1e-3 / dcount
        gbs = B / avg_s / 1e9
        tfl = F / avg_s / 1e12
        if tfl / fp64_peak >= gbs / peaks["hbm_gbs"]:
            roof = {"bound": "alu", "kernel": dom, "achieved": tfl, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": tfl / fp64_peak, "traffic": traffic_of(dom, "fp64"),
                    "peak_note": "FP64 FMA, measured in this run by sie_probe_fma (nominal 1.25 TFLOP/s)",
                    "hbm_gbs_achieved": gbs, "hbm_frac": gbs / peaks["hbm_gbs"]}
        else:
            roof = {"bound": "hbm", "kernel": dom, "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "traffic": traffic_of(dom, "fp64"),
                    "peak_note": f"HBM copy, {kind}"}
        roof.update({"algorithmic_bytes": B, "algorithmic_flops": F, "avg_launch_us": avg_s * 1e6,
                     "launches": dcount})
    # every modelled stage of the FP64 path: fraction of the FP64 FMA and HBM peaks
    stage_roofs = {}
    for k, (tms, cnt) in kern.items():
        mdl = stage_model(k, info, ne, nt, info[8], nnz_int)
        if mdl is None or cnt == 0:
            continue
        a_s = tms * 1e-3 / cnt
        stage_roofs[k] = {"avg_launch_us": round(a_s * 1e6, 2),
                          "fp64_frac": round(mdl[1] / a_s / 1e12 / fp64_peak, 4),
                          "hbm_frac": round(mdl[0] / a_s / 1e9 / peaks["hbm_gbs"], 4)}
    if graph_state & 1:
        # graph replay: nodes outside the nested loop + loop-body nodes per nested
        # iteration (upper bound: the largest iteration count of the timed loop)
        launches = args.steps * int(ginfo[17] + ginfo[18] * gstats["inner_iters_max"])
    else:
        launches = sum(c for _, c in prof.values())
    cpu = cpu_baseline(args) if not args.no_cpu and world == 1 else None  # rank 0 at N = 1 only
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "interior": args.interior, "ne": ne, "nt": nt,
                   "grid_N": info[0:3].tolist(), "fft_n": info[3:6].tolist(), "near_nnz_ext": int(info[8]),
                   "near_nnz_int": int(nnz_int), "step": "system matvec, Eq. (sys) (AEFIE, [H; c0 rho])",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "build_s": build_s, "build_ms_breakdown": info[12:16].tolist()},
        "e2e": {"value": job_value(world, ne, args.steps, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": n * 16,
                "d2h_bytes_per_step": n * 16},
        "gpu_launches": launches,
        "ms_per_step_with_stage_events": ms_prof / args.steps,
        "nested_solves": nested,
        "system_graph": {"fp64": bool(graph_state & 1), "capture_failed": bool(graph_state & 4),
                         "nodes_outside_loop": int(ginfo[17]), "nodes_per_nested_iteration": int(ginfo[18]),
                         "nested_iterations_max": int(gstats["inner_iters_max"]),
                         "note": "timed loop replays one CUDA graph per product (nested solve as a device-ended "
                                 "loop); the stage breakdown comes from the stream path with per-stage events"},
        "solves": solves,
        "solves_workload": lossy_solves,
        "batching": batching,
        "ports": ports,
        "serving": serving,
        "block_rhs": block,
        "mixed_precision": mixed_line(ne, args, ms32, prof32, mixed_err, info, peaks, kind),
        "stages_ms": {k: round(v[0], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "roofline": roof,
        "stage_rooflines": stage_roofs,
        "fma_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak, "how": "sie_probe_fma, this run"},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line, default=_jsonable))


def mixed_line(ne, args, ms32, prof, err, info, peaks, kind):
    """The complex64 path (SIE_MIXED): throughput, error vs FP64, HBM roofline of
    its dominant stage among the FFT passes, the spectral multiply and the
    exterior near-region products (8 B per complex64 value)."""
    N = info[0:3].astype(np.int64)
    n = info[3:6].astype(np.int64)
    Nx, Ny, Nz = N
    nx, ny, nz = n
    c = 8
    ne = int(ne)
    nnz_ext, ntri = int(info[8]), int(info[7])
    model = {"fft_fwd_x": (Nx * Ny * Nz + nx * Ny * Nz) * c, "fft_fwd_y": (nx * Ny * Nz + nx * ny * Nz) * c,
             "fft_fwd_z": (nx * ny * Nz + nx * ny * nz) * c, "fft_inv_z": (nx * ny * nz + nx * ny * Nz) * c,
             "fft_inv_y": (nx * ny * Nz + nx * Ny * Nz) * c, "fft_inv_x": (nx * Ny * Nz + Nx * Ny * Nz) * c,
             "specmul_sys32": (7 + 4 + 4) * nx * ny * nz * c,
             "fft_z_specmul": (11 * nx * ny * Nz + 4 * nx * ny * nz) * c,
             # complex64 exterior near values (LA, K; triangle Lphi), FP64 I-cross and vectors
             "spmv_sys": nnz_ext * (2 * c + 4) + ntri * (c + 4) + 5 * ne * 20 + 8 * ne * 16 + 6 * (n_t(info, ne)) * 16,
             # k_spmv2_c64 alone: interleaved complex64 values and columns once,
             # row pointers, the packed (H, E) read once, y (FP64) read and written
             "spmv_near_ext": nnz_ext * (2 * c + 4) + (ne + 1) * 8 + ne * 2 * c + 2 * ne * 16,
             "spmv_sys_rest": ntri * (c + 4) + 5 * ne * 20 + 4 * ne * 16 + 6 * (n_t(info, ne)) * 16}
    kern = {k: v for k, v in prof.items() if k in model}
    roof = None
    if kern:
        dom = max(kern, key=lambda k: kern[k][0])
        B = model[dom] * FFT_GRIDS.get(dom, 1)
        avg = kern[dom][0] * 1e-3 / kern[dom][1]
        roof = {"bound": "hbm", "kernel": dom, "achieved": B / avg / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": B / avg / 1e9 / peaks["hbm_gbs"], "traffic": traffic_of(dom, "mixed"),
                "peak_note": f"HBM copy, {kind}",
                "algorithmic_bytes": int(B), "avg_launch_us": avg * 1e6}
    stage_roofs = {k: {"avg_launch_us": round(v[0] * 1e3 / v[1], 2),
                       "hbm_frac": round(model[k] * FFT_GRIDS.get(k, 1) / (v[0] * 1e-3 / v[1]) / 1e9 /
                                         peaks["hbm_gbs"], 4)}
                   for k, v in kern.items() if v[1]}
    return {"value": ne * args.steps / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32 / args.steps,
            "stage_rooflines": stage_roofs,
            "dtype": "c64 grid / f64 near+Krylov", "rel_err_vs_fp64": err,
            "stages_ms": {k: round(v[0], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
            "roofline": roof}


def n_t(info, ne):
    """Triangle count of a closed mesh from its edge count (3 N_t = 2 N_e)."""
    return 2 * ne // 3


def _jsonable(o):
    if hasattr(o, "item"):
        return o.item()
    if hasattr(o, "tolist"):
        return o.tolist()
    return str(o)


def solve_stats(sie, ctx, args):
    """GMRES solves of the dielectric sphere (1,920 RWG, eps_r = 4, 3 GHz, r = 1 cm,
    equal-volume icosphere) for seeded incidence directions, to tol_outer 1e-6:
    the FP64 solve and the mixed-precision refinement (SIE_SOLVE_REFINE) on the
    same right-hand sides.  Each solve's backscatter RCS is compared with the
    Mie series; solves/s counts every solve, `ok` those within 1% of Mie that
    converged."""
    name = "dielectric-sphere-1920"
    wl = workload(name)
    ref = mie_backscatter(name)
    mesh = sie.Mesh(ctx, wl["V"], wl["T"])
    op = sie.Operator(mesh, wl["f"], wl["eps_r"], 1.0, wl["sigma"], sie.params(tol_outer=1e-6))
    rng = np.random.default_rng(7)
    dirs = []
    for i in range(args.solves):
        z = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * np.pi)
        kh = np.array([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z])
        ep = np.cross(kh, [0.3, -0.5, 0.8])
        dirs.append((kh, ep / np.linalg.norm(ep)))
    out = {"workload": name, "tol": 1e-6, "solves": args.solves, "mie_backscatter_m2": ref}
    xs = {}
    for refine in (False, True):
        lat, its, errs, conv = [], [], [], []
        for i, (kh, ep) in enumerate(dirs):
            b = op.rhs_planewave(kh, ep)
            t0 = time.perf_counter()
            x, it, rr = op.solve(b, check=False, refine=refine)
            lat.append(time.perf_counter() - t0)
            its.append(int(it[0]))
            conv.append(bool(rr[0] < 1e-6))
            errs.append(float(op.rcs(x, -kh)[0] / ref - 1.0))
            xs[(refine, i)] = x
        lat = np.array(lat)
        ok = [c and abs(e) <= 0.01 for c, e in zip(conv, errs)]
        out["refined" if refine else "fp64"] = {
            "solves_per_s": float(len(lat) / lat.sum()), "ok_solves": int(sum(ok)), "not_converged": conv.count(False),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)), "iters": its,
            "rcs_rel_err_vs_mie": errs}
    out["refined_vs_fp64"] = {
        "speedup": out["refined"]["solves_per_s"] / out["fp64"]["solves_per_s"],
        "max_rel_diff_x": max(float(np.linalg.norm(xs[(True, i)] - xs[(False, i)]) / np.linalg.norm(xs[(False, i)]))
                              for i in range(len(dirs)))}
    op.close()
    mesh.close()
    return out


def block_stats(sie, op, ne, stream, args, R=8, reps=5):
    """Exterior AIM products L0 for R right-hand sides: one block call (spectra,
    weights and near values read once) against R single-vector calls, device
    pointers, CUDA events on the library's stream."""
    import torch
    X = torch.randn(R, ne, dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(block):
        if block:
            op.matvec(sie.SIE_OP_L0, X, Y, nrhs=R)
        else:
            for r in range(R):
                op.matvec(sie.SIE_OP_L0, X[r], Y[r])

    out = {}
    for block in (True, False):
        run(block)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            run(block)
        e1.record(stream)
        torch.cuda.synchronize()
        out["block" if block else "single"] = e0.elapsed_time(e1) / reps / R
    return {"operator": "L0 (exterior AIM L, Eq. AIM_Lin)", "rhs": R, "ms_per_rhs_block": out["block"],
            "ms_per_rhs_single": out["single"], "speedup": out["single"] / out["block"]}


def lossy_solve_stats(sie, op, args, wl):
    """GMRES solves of the timed workload itself (tol_outer 1e-4, Sec. V) for
    seeded incidence directions: the FP64 solve and the mixed-precision
    refinement (SIE_SOLVE_REFINE) on the same right-hand sides; solves/s,
    latency, iterations, and each solve's backscatter RCS against the Mie
    series (ok: converged and within 1%).  One untimed warm-up solve first
    (graph capture, Krylov workspaces)."""
    ref = mie_backscatter(args.workload)
    rng = np.random.default_rng(11)
    dirs = []
    for i in range(args.lossy_solves):
        z = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * np.pi)
        kh = np.array([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z])
        ep = np.cross(kh, [0.3, -0.5, 0.8])
        dirs.append((kh, ep / np.linalg.norm(ep)))
    out = {"workload": args.workload, "tol": op_tol(sie), "solves": len(dirs), "mie_backscatter_m2": ref,
           "dense_constraint_lu_ms": float(op.info()[19])}
    for refine in (False, True):
        if dirs:
            op.solve(op.rhs_planewave(*dirs[0]), check=False, refine=refine)
        lat, its, errs, conv = [], [], [], []
        for kh, ep in dirs:
            b = op.rhs_planewave(kh, ep)
            t0 = time.perf_counter()
            x, it, rr = op.solve(b, check=False, refine=refine)
            lat.append(time.perf_counter() - t0)
            its.append(int(it[0]))
            conv.append(bool(rr[0] < op_tol(sie)))
            errs.append(float(op.rcs(x, -kh)[0] / ref - 1.0))
        lat = np.array(lat)
        out["refined" if refine else "fp64"] = {
            "solves_per_s": float(len(lat) / lat.sum()) if len(lat) else None,
            "ok_solves": int(sum(c and abs(e) <= 0.01 for c, e in zip(conv, errs))),
            "not_converged": conv.count(False), "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None, "iters": its,
            "rcs_rel_err_vs_mie": errs, "last_solve_stats": op.stats()}
    if dirs:
        out["refined_vs_fp64"] = {"speedup": out["refined"]["solves_per_s"] / out["fp64"]["solves_per_s"]}
    # one block of R right-hand sides solved in lockstep (sie_solve nrhs = R)
    R = args.lockstep_rhs
    if R > 1:
        bdirs = []
        for i in range(R):
            z = rng.uniform(-1, 1)
            ph = rng.uniform(0, 2 * np.pi)
            kh = np.array([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z])
            ep = np.cross(kh, [0.3, -0.5, 0.8])
            bdirs.append((kh, ep / np.linalg.norm(ep)))
        B = np.stack([op.rhs_planewave(kh, ep) for kh, ep in bdirs])
        for refine in (False, True):
            t0 = time.perf_counter()
            X, it, rr = op.solve(B, nrhs=R, check=False, refine=refine)
            dt = time.perf_counter() - t0
            errs = [float(op.rcs(X[q], -bdirs[q][0])[0] / ref - 1.0) for q in range(R)]
            conv = [bool(v < op_tol(sie)) for v in rr]
            out[("refined" if refine else "fp64") + "_lockstep"] = {
                "rhs": R, "wall_s": dt, "solves_per_s": R / dt, "iters": int(it.max()),
                "ok_solves": int(sum(c and abs(e) <= 0.01 for c, e in zip(conv, errs))),
                "rcs_rel_err_vs_mie_max": float(np.abs(errs).max())}
        if dirs:
            out["refined_lockstep_vs_fp64"] = {
                "speedup": out["refined_lockstep"]["solves_per_s"] / out["fp64"]["solves_per_s"],
                "note": "solves/s of the mixed-precision refinement with lockstep blocks over the plain FP64 "
                        "path solving one right-hand side at a time, same workload and tolerance"}
    return out


def batching_stats(sie, ctx, args):
    """Batching (the batching configuration, scaled to one GPU for a minute):
    three meshes of uneven sizes (a 1,280-triangle sphere, a 768-triangle
    cube, a 320-triangle sphere), two frequencies each, args.batch_rhs
    plane waves per (mesh, frequency).  Each set is solved one right-hand
    side at a time (FP64) and in lockstep blocks of 8 (FP64 and the
    mixed-precision refinement) on the same operator; solves/s over all
    sets, and the largest difference of the lockstep solutions from the
    one-at-a-time ones."""
    from synth import box, icosphere
    rng = np.random.default_rng(23)
    meshes = [("sphere-1280", icosphere(3, 5e-3, equal_volume=True)),
              ("cube-768", box((8e-3, 8e-3, 8e-3), (8, 8, 8))),
              ("sphere-320", icosphere(2, 2e-3, equal_volume=True))]
    mats = [(3e9, 4.0, 0.0), (10e9, 1.0, 5.8e7)]
    tot = {"fp64_sequential": 0.0, "fp64_lockstep": 0.0, "refined_lockstep": 0.0}
    nrhs, worst, conv, sets = 0, 0.0, 0, []
    for name, (V, T) in meshes:
        mesh = sie.Mesh(ctx, V, T)
        for f, er, sg in mats:
            op = sie.Operator(mesh, f, er, 1.0, sg, sie.params())
            dirs = []
            for _ in range(args.batch_rhs):
                z = rng.uniform(-1, 1)
                ph = rng.uniform(0, 2 * np.pi)
                kh = np.array([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z])
                ep = np.cross(kh, [0.3, -0.5, 0.8])
                dirs.append((kh, ep / np.linalg.norm(ep)))
            B = np.stack([op.rhs_planewave(kh, ep) for kh, ep in dirs])
            op.solve(B[:2], nrhs=2, check=False)  # graph capture and workspaces, untimed
            t0 = time.perf_counter()
            Xs, _, _ = op.solve(B, nrhs=len(B), sequential=True, check=False)
            t1 = time.perf_counter()
            Xb, itb, rrb = op.solve(B, nrhs=len(B), check=False)
            t2 = time.perf_counter()
            Xr, itr, rrr = op.solve(B, nrhs=len(B), refine=True, check=False)
            t3 = time.perf_counter()
            tot["fp64_sequential"] += t1 - t0
            tot["fp64_lockstep"] += t2 - t1
            tot["refined_lockstep"] += t3 - t2
            nrhs += len(B)
            conv += int(sum(rrb < op_tol(sie))) + int(sum(rrr < op_tol(sie)))
            worst = max(worst, max(float(np.linalg.norm(Xb[q] - Xs[q]) / np.linalg.norm(Xs[q])) for q in range(len(B))))
            sets.append({"mesh": name, "f_hz": f, "eps_r": er, "sigma": sg, "unknowns": mesh.ne + mesh.nt,
                         "iters_lockstep": int(itb.max()), "iters_refined": int(itr.max())})
            op.close()
        mesh.close()
    out = {"sets": sets, "rhs_per_set": args.batch_rhs, "solves": nrhs, "converged_of_2x": conv,
           "max_rel_diff_lockstep_vs_sequential": worst}
    for k, v in tot.items():
        out[k + "_solves_per_s"] = nrhs / v
    out["lockstep_speedup_fp64"] = tot["fp64_sequential"] / tot["fp64_lockstep"]
    out["refined_lockstep_vs_fp64_sequential"] = tot["fp64_sequential"] / tot["refined_lockstep"]
    out["not_built"] = "frequency points in one graph launch; an autotuner; tensor-core near blocks"
    return out


def ports_stats(sie, ctx, args):
    """Ports (the delta-gap model of sie_port_*), two small interconnect-style
    structures of copper (structured meshes, 2 um cells):
    * a bar, 40 x 4 x 4 um (336 triangles / 504 RWG), with two ports across
      its cross-section at x = -10 um and +10 um;
    * two parallel bars of that size 4 um apart (two objects, 672 triangles),
      one port across the middle of each.
    At each frequency of args.port_freqs: the admittance matrix (all ports in
    one lockstep solve block, tolerance 1e-4 as in Sec. V) and S (50 ohm),
    with the near-region-only interior and with the surface impedance
    comparator.  Reports the time per admittance matrix (over the solves that
    reached the tolerance; the others, stopped at 300 iterations, are counted
    and flagged) and the reciprocity |Y12 - Y21| / |Y12|."""
    from synth import box
    Va, Ta = box((40e-6, 4e-6, 4e-6), (20, 2, 2), center=(0.0, -4e-6, 0.0))
    Vb, Tb = box((40e-6, 4e-6, 4e-6), (20, 2, 2), center=(0.0, 4e-6, 0.0))
    V1, T1 = box((40e-6, 4e-6, 4e-6), (20, 2, 2))
    structures = [
        ("bar, 2 ports", V1, T1, None,
         [((-10e-6, 0.0, 0.0), (1.0, 0.0, 0.0), 8e-6), ((10e-6, 0.0, 0.0), (1.0, 0.0, 0.0), 8e-6)]),
        ("two coupled bars, 1 port each", np.vstack([Va, Vb]), np.vstack([Ta, Tb + len(Va)]),
         np.concatenate([np.zeros(len(Ta), np.int32), np.ones(len(Tb), np.int32)]),
         [((0.0, -4e-6, 0.0), (1.0, 0.0, 0.0), 3e-6), ((0.0, 4e-6, 0.0), (1.0, 0.0, 0.0), 3e-6)]),
    ]
    rows, t_conv, n_conv, n_stalled = [], 0.0, 0, 0
    for sname, V, T, obj, pts in structures:
        mesh = sie.Mesh(ctx, V, T, obj=obj)
        try:
            if obj is not None:
                for o in range(2):
                    mesh.set_material(o, 1.0, 1.0, 5.8e7)
            for model, name in ((sie.SIE_GIBC, "gibc"), (sie.SIE_SIBC, "sibc")):
                for f in args.port_freqs:
                    # iteration cap 300 (the converging cases need at most 177)
                    op = sie.Operator(mesh, f * 1e9, 1.0, 1.0, 5.8e7, sie.params(interior_model=model, maxit=300))
                    try:
                        op.port_admittance(pts, check=False)  # workspaces and graph, untimed
                        t0 = time.perf_counter()
                        Y, it, rr = op.port_admittance(pts, check=False)
                        dt = time.perf_counter() - t0
                        converged = bool(np.all(rr <= op_tol(sie)))
                        if converged:
                            t_conv += dt
                            n_conv += 1
                        else:
                            n_stalled += 1
                        S = sie.port_sparams(Y, 50.0)
                        rows.append({"structure": sname, "interior": name, "f_ghz": f,
                                     "near_only": bool(op.info()[9] == 1.0),
                                     "Y11": [Y[0, 0].real, Y[0, 0].imag], "Y21": [Y[1, 0].real, Y[1, 0].imag],
                                     "S11": [S[0, 0].real, S[0, 0].imag], "S21": [S[1, 0].real, S[1, 0].imag],
                                     "reciprocity": float(abs(Y[0, 1] - Y[1, 0]) / abs(Y[0, 1])),
                                     "iters": it.tolist(), "relres": rr.tolist(), "converged": converged,
                                     "ms": 1e3 * dt})
                    finally:
                        op.close()
        finally:
            mesh.close()
    return {"workload": "copper bar 40x4x4 um (336 triangles, 2 ports); two such bars 4 um apart "
                        "(672 triangles, 1 port each)", "rows": rows,
            "ms_per_admittance_converged": 1e3 * t_conv / max(n_conv, 1), "converged": n_conv,
            "stalled_at_maxit": n_stalled}


def serve_catalogue():
    """The serving trace's operators: (name, radius, f, eps_r, sigma, level,
    Mie backscatter) as drawn and evaluated by tests/golden/make_mie_backscatter.py."""
    path = os.path.join(ROOT, "tests", "golden", "mie_backscatter.txt")
    out = []
    for line in open(path):
        f = line.split()
        if f and f[0].startswith("serve-"):
            out.append((f[0], float(f[1]), float(f[2]), float(f[3]), float(f[4]), int(f[0][-1]), float(f[5])))
    return out


def serving_stats(args):
    """Serving trace (the serving configuration, scaled to one GPU for
    minutes): args.serve_requests requests with Poisson arrivals at
    args.serve_rate per second, each on one of the catalogue's operators
    (uniform) with 1 to 4 plane waves (backscatter), through the request
    loop (paper_2003_11679_gb300/serve.py: two slots, shared resident
    operator cache, cross-request batching into lockstep solves).  Two traces
    on one server: `cold` starts with an empty cache (the catalogue's operator
    builds fall in the trace), `warm` follows with new arrivals on the
    resident operators.  Latency is per request from its arrival; solves/s
    counts right-hand sides over the trace's wall time; each solve's RCS is
    compared with the Mie series."""
    from paper_2003_11679_gb300.serve import Request, Server
    from synth import icosphere
    cat = serve_catalogue()
    rng = np.random.default_rng(17)
    meshes = {c[0]: icosphere(c[5], c[1], equal_volume=True) for c in cat}

    def draw():
        reqs, arrivals, t = [], [], 0.0
        for i in range(args.serve_requests):
            t += rng.exponential(1.0 / args.serve_rate)
            c = cat[rng.integers(len(cat))]
            k = int(rng.integers(1, 5))
            khs, eps = [], []
            for _ in range(k):
                z = rng.uniform(-1, 1)
                ph = rng.uniform(0, 2 * np.pi)
                kh = np.array([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z])
                ep = np.cross(kh, [0.3, -0.5, 0.8])
                khs.append(kh)
                eps.append(ep / np.linalg.norm(ep))
            V, T = meshes[c[0]]
            reqs.append((Request(V, T, c[2], c[3], c[4], np.array(khs), np.array(eps), -np.array(khs)), c))
            arrivals.append(t)
        return reqs, arrivals

    def trace(srv, reqs, arrivals):
        before = dict(srv.counters)
        nlat0 = len(srv._lat)
        errs, res, nrhs, failed = [], [], 0, []
        t0 = time.perf_counter()
        futs = []
        for (r, c), ta in zip(reqs, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            futs.append((srv.submit(r), r, c))
        for f, r, c in futs:
            try:
                out = f.result(timeout=1800)
            except Exception as e:  # reported in the line, the trace goes on
                failed.append(f"{c[0]}: {type(e).__name__}: {e}"[:200])
                continue
            rcs = np.atleast_2d(out["rcs"])
            for q in range(r.nrhs):
                errs.append(float(rcs[q, q] / c[6] - 1.0))  # backscatter: rhat_q = -khat_q
            res.extend(np.atleast_1d(out["relres"]).tolist())
            nrhs += r.nrhs
        wall = time.perf_counter() - t0
        lat = np.array(srv._lat[nlat0:])
        cnt = {k: srv.counters.get(k, 0) - before.get(k, 0) for k in ("built", "reused", "batched")}
        ae = np.abs(errs) if errs else np.array([np.nan])
        return {"requests": len(reqs), "right_hand_sides": nrhs, "wall_s": wall, "solves_per_s": nrhs / wall,
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None, **cnt,
                "converged": int(sum(v < 1e-4 for v in res)),
                "rcs_rel_err_vs_mie_p50": float(np.median(ae)), "rcs_rel_err_vs_mie_max": float(ae.max()),
                "within_1pct": int((ae <= 0.01).sum()), "failed_requests": failed}

    with Server(slots=2) as srv:
        cold = trace(srv, *draw())
        warm = trace(srv, *draw())
    return {"rate_per_s": args.serve_rate, "slots": 2, "operators": len(cat), "cold": cold, "warm": warm,
            "note": "catalogue = tests/golden/mie_backscatter.txt serve-* rows (spheres, level 2-3 meshes, "
                    "the serving configuration's sigma, eps_r and frequency ranges)"}


def op_tol(sie):
    return sie.params().tol_outer


class OracleStep:
    """One step of the oracle on a bounded sample of a workload: the system
    product of Eq. (sys) in its AIM form (oracle/system.AimGIBC: exterior AIM
    products with their near corrections, near-region-only interior Z' by a
    sparse LU; AIM interior for a dielectric) on a level-2 icosphere of the
    same radius, material and exterior grid.  Set-up (near-region integrals,
    factorisation) is not part of the step."""

    def __init__(self, wl):
        from oracle import aim, system
        from oracle.rwg import Mesh
        from synth import cn_vector, icosphere
        V, T = icosphere(2, wl["radius"])
        self.m = Mesh(V, T)
        mfull = Mesh(wl["V"], wl["T"])
        gfull = aim.grid_params(mfull, M=2, grid_n=wl["grid_n"] or None)
        # the sample keeps the workload's grid spacing, extent and FFT size
        g = aim.grid_params(self.m, M=2, h=gfull.h)
        ki = system.k_medium(wl["f"], wl["eps_r"], wl["sigma"])
        delta = 1.0 / abs(ki.imag) if ki.imag != 0 else np.inf
        near = 5 * delta <= (g.Rnear - g.M) * g.h
        self.S = system.AimGIBC(self.m, wl["f"], wl["eps_r"], wl["sigma"], g,
                                interior="near" if near else "aim", cutoff=5 * delta if near else None)
        self.H, self.rho = cn_vector(self.m.ne, 1), cn_vector(self.m.nt, 2)
        self.grid_N, self.full_N = [int(v) for v in g.N], [int(v) for v in gfull.N]

    def __call__(self):
        return self.S.apply(self.H, self.rho)

    def describe(self, ne_full):
        return (f"oracle system product of Eq. (sys) (AIM exterior with near terms, near-only interior Z' by sparse "
                f"LU) on a 320-triangle sample of the same sphere, material and exterior grid (N {self.grid_N} vs "
                f"{self.full_N} of the full mesh: the same FFT size); value = {ne_full} RWG unknowns / step time, an "
                f"upper bound of the oracle's full-size throughput (its grid part has the full size, its near and "
                f"interior parts are smaller); numpy/scipy kernels, single-threaded")


def cpu_baseline(args):
    """The oracle's step (OracleStep) on the host: one warm-up, median of >= 5."""
    wl = workload(args.workload)
    step = OracleStep(wl)
    step()
    ts = []
    t_end = time.perf_counter() + args.cpu_seconds
    while len(ts) < 5 or (time.perf_counter() < t_end and len(ts) < 50):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    med = float(np.median(ts))
    model, ncpu = cpu_info()
    ne_full = 3 * len(wl["T"]) // 2
    return {"value": ne_full / med, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": step.describe(ne_full),
            "median_step_s": med, "steps": len(ts), "cpu_model": model, "host_cpus": ncpu,
            "sample_rwg": step.m.ne, "sample_value": step.m.ne / med}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args.workload)
    t_wall = time.perf_counter()
    step = OracleStep(wl)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    ne_full = 3 * len(wl["T"]) // 2
    value = ne_full * args.steps / dt
    model, ncpu = cpu_info()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": step.describe(ne_full), "value": value,
                             "cpu_model": model, "host_cpus": ncpu},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_wall}
    print(json.dumps(line, default=_jsonable))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lossy-sphere-30720")
    ap.add_argument("--cpu-seconds", type=float, default=30.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--solves", type=int, default=4)
    ap.add_argument("--lossy-solves", type=int, default=3)
    ap.add_argument("--lockstep-rhs", type=int, default=8)
    ap.add_argument("--batch-rhs", type=int, default=16)
    ap.add_argument("--port-freqs", type=float, nargs="*", default=[50.0, 100.0, 200.0],
                    help="frequencies (GHz) of the ports leg; none to skip it")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--interior", default="gibc", choices=["gibc", "sibc"],
                    help="interior model of the timed operator (sibc: the surface impedance comparator)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
