#!/usr/bin/env python
"""Benchmark of the KFBI Stokes solver on GB300.

One step = one full kfbim_solve (Alg. 1): the volume interface solve for the
right-hand side, GMRES to 1e-10 on the BIE (one interface solve per
iteration) and the final interior-field interface solve, on the star
workload r = 0.5 + 0.1 sin(3 theta) cos(4 phi) in [-1, 1]^3 at N = 128 with
the manufactured Stokes data.  Inputs are resident in HBM when the timed
region starts; the L2 is flushed (a 512 MiB write) before every step, outside
the per-step CUDA events.

Printed JSON line (rank 0): value = solves/s over all ranks (MIXED precision),
the FP64 path's solves/s beside it, the relative difference of the MIXED
density from the FP64 one, the roofline of the dominant kernel (the FP32
transform passes, timed with CUDA events around each launch in a second run
of the same steps), the oracle CPU baseline, e2e through kfbim_solve_host with
host buffers, the kernel-launch count and the SM clocks sampled during the
timed region; beside them, the autotuner's choice of transform kernels, one
adjoint (gradient) solve on the same data, and a batch of 16 instances in one
kfbim_solve_batch call against the same instances solved one at a time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kfbim|reference]
Multi-GPU (torchrun): replicas only, every rank solves its own instance, no
collective on the data path ("scaling": "weak").
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import kfbim_inputs as ki  # noqa: E402

METRIC = "Stokes BIE solves/s at 128^3 (mixed vs FP64, rel err ≤1e-8); HBM GB/s"
WORKLOAD = "star128"
WORKLOAD_DESC = ("Stokes interior Dirichlet on the star r=0.5+0.1 sin(3theta) cos(4phi) in [-1,1]^3, "
                 "MAC grid 128^3, mu=1, manufactured u=(sin x cos y cos z, -cos x sin y cos z, 0), "
                 "p=sin(x+y+z), GMRES tol 1e-10")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kfbim", choices=["kfbim", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--refine-tol", type=float, default=None, help="MIXED refinement tolerance")
    ap.add_argument("--inner-tol", type=float, default=None, help="MIXED inner FP32 CG tolerance")
    ap.add_argument("--relax", type=float, default=None,
                    help="MIXED inexact-GMRES relaxation factor (library default 0.1; 0 = off)")
    ap.add_argument("--transforms", default="auto", choices=["auto", "fft", "tensor", "staged"],
                    help="kernels of the FP32 axis passes (auto: the setup-time autotuner's choice)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (gradient) leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 256^3 FP32 forward leg")
    ap.add_argument("--batch", type=int, default=16,
                    help="instances of the batched leg (kfbim_solve_batch); 0 skips it")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-solve", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--interface-solves", type=int, default=None,
                    help="interface solves per solve for the reference arm's scaling "
                         "(default: the workload's count in INTERFACE_SOLVES)")
    return ap.parse_args()


# Interface solves of one solve of each workload (GMRES iterations plus the
# right-hand-side and final-field solves), as the GPU solves report them in
# their stats (FP64 and MIXED alike): the reference arm times one oracle matvec
# and scales it by this count.
INTERFACE_SOLVES = {"sphere32": 18, "star128": 61}


# ------------------------------------------------------------ oracle sample
def oracle_sample(workload, reps, per_solve):
    """Time the oracle (single thread) on `reps` matvecs of the workload."""
    from oracle import kfbim as okfbim
    geom, grid = ki.WORKLOADS[workload]
    s = okfbim.Setup(geom, grid)
    phi = ki.random_density(s.n, seed=0)
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        s.apply(phi)
        times.append(time.perf_counter() - t)
    t_mv = statistics.median(times)
    return {"matvec_s": t_mv, "times": times, "value": 1.0 / (t_mv * per_solve)}


def oracle_full_solve(workload):
    """One complete oracle solve (Alg. 1: right-hand-side volume solve, GMRES
    to 1e-10, final fields) of a workload's manufactured data, timed."""
    from oracle import kfbim as okfbim
    geom, grid = ki.WORKLOADS[workload]
    t0 = time.perf_counter()
    s = okfbim.Setup(geom, grid)
    t_setup = time.perf_counter() - t0
    x = s.cp.xyz
    g = ki.stokes_velocity(x)[np.arange(s.cp.n), s.cp.comp - 1][s.primary]
    fy = ki.stokes_forcing(x)
    ff = [ki.stokes_forcing(s.grid.node_xyz(c, s.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    t0 = time.perf_counter()
    sol = s.solve(g, fy, ff)
    t = time.perf_counter() - t0
    return {"workload": workload, "solve_s": round(t, 3), "setup_s": round(t_setup, 3),
            "solves_per_s": round(1.0 / t, 5), "gmres_iters": int(sol["iters"]),
            "value_kind": "timed", "threads": 1}


def run_oracle_solve_subprocess(workload):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-solve", "--workload", workload],
                       capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle solve failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_parallel(workload, procs):
    """`procs` single-threaded oracle processes, each one full solve of the
    workload, started together on the host's cores: aggregate solves/s over
    the wall time of the slowest."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-solve", "--workload", workload]
    t0 = time.perf_counter()
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    outs = [p.communicate() for p in ps]
    wall = time.perf_counter() - t0
    if any(p.returncode != 0 for p in ps):
        raise RuntimeError("parallel oracle solve failed:\n" + outs[0][1][-2000:])
    return {"workload": workload, "processes": procs, "wall_s": round(wall, 3),
            "solves_per_s": round(procs / wall, 4), "value_kind": "timed",
            "sample": "%d concurrent single-threaded full oracle solves of %s" % (procs, workload)}


def run_oracle_subprocess(workload, reps, per_solve):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload",
                        workload, "--steps", str(reps), "--interface-solves", str(per_solve)],
                       capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PASS_SOURCES = {"fft": ("transforms.cuh", "transforms2.cuh"),
                 "tensor": ("transforms.cuh", "transforms2.cuh", "tc_pass.cuh")}


def kernel_source_hash(kind="fft"):
    h = hashlib.sha256()
    for f in PASS_SOURCES[kind]:
        h.update(open(os.path.join(ROOT, "paper_2303_04992_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def ncu_traffic(workload, kind="fft"):
    """DRAM bytes per launch of the FP32 transform pass (FFT or tensor-core
    kernel) from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    name = "axis_pass_fp32_%s.md" if kind == "fft" else "tc_pass_fp32_%s.md"
    p = os.path.join(ROOT, "profiles", name % workload)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel_source_sha256_12:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash(kind):
        return None
    return float(t.group(1))


# Algorithmic bytes of the hot path by a three-pass byte model of the Schur
# apply (FP32 values, b = 4):
# one Schur apply S d moves 20 N^3 b (three passes over three fields, read and
# written, plus d read and q written); the CG vector updates 7 N^3 b (x, r, d,
# q read; x, r, d written); one CG iteration 27 N^3 b.  The middle pass of
# the Schur apply (forward transform, spectral weight, inverse transform of
# the three fields) is 6 N^3 b of the 20.
MODEL_B = 4
MODEL_SCHUR_VALUES = 20
MODEL_CG_VECTOR_VALUES = 7
MODEL_MIDDLE_PASS_VALUES = 6
SLAB_CLASSES = ("cg_zfwd", "cg_xy", "cg_zinv", "cg_update")


def ncu_traffic_slab(workload):
    """DRAM bytes per launch of k_cg_xy from the committed ncu summary, if it
    was taken on the current slab source (else None)."""
    p = os.path.join(ROOT, "profiles", "cg_xy_%s.md" % workload)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    h = hashlib.sha256()
    for f in ("slab.cuh", "cg_common.cuh", "transforms2.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2303_04992_gb300", "csrc", f), "rb").read())
    m = re.search(r"kernel_source_sha256_12:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != h.hexdigest()[:12]:
        return None
    return float(t.group(1))


def roofline_line(kernels, kprof, N3, cg_iters, args, peak, peak_kind):
    """The roofline object of the bench line.  Dominant kernel: the one with
    the largest share of the step.  For the slab CG the algorithmic bytes per
    launch are the byte model's figure for the work the kernel does: k_cg_xy
    does the middle pass of the Schur apply on all three terms (6 N^3 b); the
    whole CG iteration (three kernels, plus each run's closing update spread
    over its iterations) is reported beside it against 27 N^3 b."""
    dom = max(kernels, key=lambda k: kernels[k]["share_of_step"])
    kd = kernels[dom]
    line = {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_kind,
            "kernel": dom, "avg_launch_us": kd["avg_launch_us"], "launches_per_step": kd["launches_per_step"],
            "share_of_step": kd["share_of_step"], "build_bytes_per_launch": kd["build_bytes_per_launch"],
            "achieved_build_bytes": kd["achieved_gbs_build_bytes"]}
    if dom == "cg_xy":
        model = MODEL_MIDDLE_PASS_VALUES * N3 * MODEL_B
        line["model"] = "three-pass byte model: middle pass of S d on three fields, 6 N^3 b, b = 4"
        line["traffic"] = ncu_traffic_slab(args.workload)
    elif dom in ("transform_fp32", "transform_fp64"):
        # one one-axis pass of one field: 2 N^3 b per job, at the launch's jobs
        model = kd["build_bytes_per_launch"]
        line["model"] = "one-axis pass: N^3 values read and written per job"
        line["traffic"] = ncu_traffic(args.workload, "fft")
    else:
        model = kd["build_bytes_per_launch"]
        line["model"] = "values read and written once"
        line["traffic"] = None
    achieved = model / (kd["avg_launch_us"] * 1e-6) / 1e9
    line["algorithmic_bytes_per_launch"] = model
    line["achieved"] = round(achieved, 1)
    line["frac"] = round(achieved / peak, 4)
    if all(k in kprof and kprof[k][1] for k in SLAB_CLASSES) and cg_iters:
        ms_cg = sum(kprof[k][0] for k in SLAB_CLASSES)
        it_us = ms_cg / cg_iters * 1e3
        bytes_it = (MODEL_SCHUR_VALUES + MODEL_CG_VECTOR_VALUES) * N3 * MODEL_B
        line["cg_iteration"] = {"us": round(it_us, 3), "model_bytes": bytes_it,
                                "achieved": round(bytes_it / (it_us * 1e-6) / 1e9, 1),
                                "frac": round(bytes_it / (it_us * 1e-6) / 1e9 / peak, 4),
                                "model": "three-pass byte model: 27 N^3 b per CG iteration (S d 20, vectors 7)"}
    return line


def golden_error(workload, phi):
    """Relative max-norm difference of a density from the FP64 oracle's
    solve of the workload (tests/golden, written by a script that calls only
    the oracle), or None when no stored solve exists."""
    p = os.path.join(ROOT, "tests", "golden", "%s_solve.npz" % workload)
    if not os.path.exists(p):
        return None
    want = np.load(p)["phi"]
    if len(want) != len(phi):
        return None
    return float(np.abs(phi - want).max() / np.abs(want).max())


def inputs(solver, geom, grid, navier=False):
    """Manufactured data (Stokes velocity, or the Lame displacement for the
    Navier workload): g at the primary points, f at all points and on the face
    grids (host numpy)."""
    vel = ki.lame_displacement if navier else ki.stokes_velocity
    frc = ki.lame_forcing if navier else ki.stokes_forcing
    xyz, comp, _, prim = solver.points()
    rows = np.arange(len(comp))
    g = vel(xyz)[rows, comp - 1][prim]
    fpts = frc(xyz).T.copy()
    N, lo, h = solver.N, solver.lo, solver.h
    idx = np.arange(N)
    fg = []
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                              lo + (idx + off[0]) * h, indexing="ij")      # [k, j, i]
        fg.append(frc(np.stack([X, Y, Z], -1))[..., c - 1].ravel())
    return g, fpts, np.concatenate(fg)


def host_cpu():
    """The host the oracle baseline runs on: architecture, logical CPUs and,
    where /proc/cpuinfo names it, the CPU model (x86 "model name", Arm
    implementer/part codes)."""
    import platform
    info = {"machine": platform.machine(), "logical_cpus": os.cpu_count()}
    try:
        with open("/proc/cpuinfo") as f:
            fields = {}
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
        if fields.get("model name"):
            info["model"] = fields["model name"]
        elif fields.get("CPU part"):
            info["model"] = "implementer %s part %s" % (fields.get("CPU implementer", "?"), fields["CPU part"])
    except OSError:
        pass
    return info


def job_throughput(total_ms, steps, dist=None, device="cpu"):
    """Whole-job throughput of replicas: every rank solved `steps` instances
    in total_ms of its own; the job time is the max over ranks (barrier first)
    and the value counts the instances of all ranks.  Returns (value, max_ms)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_initialized():
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    total = float(t.item())
    return world * steps / (total / 1e3), total


def adjoint_leg(solver, args, flush, stream, dev):
    """dL/dg by kfbim_solve_adjoint for L = 1/2 |u - u_t|^2 over the Omega face
    nodes (u from the bench's forward solve, u_t = 0.8 x the manufactured
    velocity), timed like the forward steps."""
    import torch
    N, lo, h = solver.N, solver.lo, solver.h
    idx = np.arange(N)
    mask, tgt = [], []
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                              lo + (idx + off[0]) * h, indexing="ij")
        tgt.append(0.8 * ki.stokes_velocity(np.stack([X, Y, Z], -1))[..., c - 1].ravel())
        mask.append(solver.sides(c).ravel().astype(np.float64))
    mask = torch.from_numpy(np.concatenate(mask)).to(dev)
    tgt = torch.from_numpy(np.concatenate(tgt)).to(dev)
    g_h, fpts_h, fgrid_h = inputs(solver, None, None)
    phi = torch.zeros(solver.n_primary, dtype=torch.float64, device=dev)
    u = torch.zeros(3 * N ** 3, dtype=torch.float64, device=dev)
    p = torch.zeros(N ** 3, dtype=torch.float64, device=dev)
    solver.solve(torch.from_numpy(g_h).to(dev), phi, torch.from_numpy(fpts_h).to(dev),
                 torch.from_numpy(fgrid_h).to(dev), u, p)
    ubar = mask * (u - tgt)
    gbar = torch.zeros_like(phi)
    solver.solve_adjoint(ubar, gbar)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 2))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
    for k in range(steps):
        flush.zero_()
        ev[2 * k].record(stream)
        solver.solve_adjoint(ubar, gbar)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)) / steps
    st = solver.last_stats
    return {"gradient_solves_per_s": round(1e3 / ms, 4), "ms_per_gradient": round(ms, 2),
            "gmres_iters": st["gmres_iters"], "interface_solves": st["interface_solves"],
            "gmres_residual": st["gmres_residual"], "api": "kfbim_solve_adjoint",
            "loss": "1/2 |u - 0.8 u_exact|^2 over the Omega face nodes", "steps": steps}


def batch_inputs(solver, B):
    """B boundary-data instances on the solver's geometry: seeded
    divergence-free harmonic fields (solid-harmonic degree <= 6, N(0,1)/(1+l)^2
    coefficients), f = 0; (B, n_primary) host array."""
    xyz, comp, _, prim = solver.points()
    rows = np.arange(len(comp))
    return np.stack([ki.harmonic_curl_field(1000 + b)(xyz)[rows, comp - 1][prim] for b in range(B)])


def batch_leg(solver, args, flush, stream, dev):
    """B instances in one kfbim_solve_batch call per step, against the same B
    instances solved one kfbim_solve call at a time."""
    import torch
    B = args.batch
    g = torch.from_numpy(batch_inputs(solver, B)).to(dev)
    phi = torch.zeros((B, solver.n_primary), dtype=torch.float64, device=dev)
    solver.solve_batch(g, phi)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 2))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
    for k in range(steps):
        flush.zero_()
        ev[2 * k].record(stream)
        solver.solve_batch(g, phi)
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)) / steps
    st = solver.last_stats
    phi_b = phi.cpu().numpy()
    # the same instances one at a time
    one = torch.zeros(solver.n_primary, dtype=torch.float64, device=dev)
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(2 * B)]
    diff = 0.0
    for b in range(B):
        flush.zero_()
        ev1[2 * b].record(stream)
        solver.solve(g[b], one)
        ev1[2 * b + 1].record(stream)
        diff = max(diff, float((one - phi[b]).abs().max() / one.abs().max()))
    torch.cuda.synchronize()
    ms1 = sum(ev1[2 * b].elapsed_time(ev1[2 * b + 1]) for b in range(B))
    return {"instances": B, "solves_per_s": round(B * 1e3 / ms, 4), "ms_per_batch": round(ms, 2),
            "single_solves_per_s": round(B * 1e3 / ms1, 4), "speedup_vs_single": round(ms1 / ms, 3),
            "gmres_iters": [s["gmres_iters"] for s in st], "kernel_launches": st[0]["kernel_launches"],
            "max_rel_diff_vs_single": diff, "phi_max": float(np.abs(phi_b).max()),
            "data": "seeded divergence-free solid-harmonic fields (degree <= 6), f = 0",
            "api": "kfbim_solve_batch", "steps": steps}


def c4_grids_leg(args, flush, stream, dev):
    """Config C4's other grids: the batch of the batched leg (star, seeded
    solid-harmonic boundary data) on star64 and star96, one kfbim_solve_batch
    call per grid (one context per grid size)."""
    import torch
    from paper_2303_04992_gb300 import MIXED, Solver
    out = {}
    for n in (64, 96):
        s = Solver(ki.star(), ki.grid(n), precision=MIXED)
        B = args.batch
        g = torch.from_numpy(batch_inputs(s, B)).to(dev)
        phi = torch.zeros((B, s.n_primary), dtype=torch.float64, device=dev)
        s.solve_batch(g, phi)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        s.solve_batch(g, phi)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = s.last_stats
        out["star%d" % n] = {"instances": B, "solves_per_s": round(B * 1e3 / ms, 4), "ms_per_batch": round(ms, 2),
                             "gmres_iters_max": max(x["gmres_iters"] for x in st),
                             "slab_cg": n in (32, 64, 128)}
        s.close()
    return out


def large_fp32_leg(args, flush, stream, dev, peak, peak_kind):
    """The FP32 forward solve at 256^3 on the star (one FP32 grid solve per
    matvec, no refinement), the manufactured forced Stokes pair as in the
    main workload: solves/s, and the one-axis transform passes against the
    measured HBM bandwidth.  At 256^3 one FP32 field is 67 MB and a pass of
    three fields moves 402 MB, three times the L2, so the passes stream from
    HBM: the HBM-bound roofline run of the transforms."""
    import torch
    from paper_2303_04992_gb300 import FP32, Solver
    geom, grid = ki.star(), ki.grid(256)
    t0 = time.perf_counter()
    s = Solver(geom, grid, precision=FP32)
    setup_s = time.perf_counter() - t0
    g_h, fpts_h, fgrid_h = inputs(s, geom, grid)
    g, fpts, fgrid = (torch.from_numpy(a).to(dev) for a in (g_h, fpts_h, fgrid_h))
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device=dev)
    s.solve(g, phi, fpts, fgrid)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record(stream)
    s.solve(g, phi, fpts, fgrid)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = dict(s.last_stats)
    s.profile(True)
    s.solve(g, phi, fpts, fgrid)
    kprof = s.profile_kernels()
    s.profile(False)
    s.close()
    ms_x, n_x, b_x = kprof["transform_fp32"]
    achieved = b_x / (ms_x * 1e-3) / 1e9
    return {"workload": "star256 (r = 0.5 + 0.1 sin 3theta cos 4phi, 256^3, [-1,1]^3)", "precision": "fp32",
            "solves_per_s": round(1e3 / ms, 4), "ms_per_solve": round(ms, 2), "setup_s": round(setup_s, 2),
            "gmres_iters": st["gmres_iters"], "cg_iters": st["cg_iters"],
            "transform_roofline": {"bound": "hbm", "kernel": "k_axis_pass2 (N = 256)", "launches": n_x,
                                   "avg_launch_us": round(ms_x / n_x * 1e3, 2),
                                   "bytes_per_launch": round(b_x / n_x), "achieved": round(achieved, 1),
                                   "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                                   "peak_source": peak_kind,
                                   "model": "every job reads and writes its field once (N^3 values each)",
                                   "share_of_solve": round(ms_x / ms, 3)},
            "api": "kfbim_solve", "steps": 1}


# -------------------------------------------------------------- main arms
def main_kfbim(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2303_04992_gb300 import FP64, MIXED, Solver, build
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    geom, grid = ki.WORKLOADS[args.workload]
    navier = args.workload in ki.NAVIER_WORKLOADS
    pde = {"mu": ki.LAME_MU, "lam": ki.LAME_LAMBDA} if navier else {}
    dev = torch.device("cuda", local)
    mixed_opts = {}
    if args.refine_tol is not None:
        mixed_opts["refine_tol"] = args.refine_tol
    if args.inner_tol is not None:
        mixed_opts["inner_tol"] = args.inner_tol
    if args.relax is not None:
        mixed_opts["relax"] = args.relax
    mixed_opts["transforms"] = {"auto": 0, "fft": 1, "tensor": 2, "staged": 3}[args.transforms]
    solver = Solver(geom, grid, precision=MIXED, **mixed_opts, **pde)
    g_h, fpts_h, fgrid_h = inputs(solver, geom, grid, navier)
    g = torch.from_numpy(g_h).to(dev)
    fpts = torch.from_numpy(fpts_h).to(dev)
    fgrid = torch.from_numpy(fgrid_h).to(dev)
    phi = torch.zeros(solver.n_primary, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        solver.solve(g, phi, fpts, fgrid)
    torch.cuda.synchronize()

    def timed(steps, profile=False):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        stats = []
        if profile:
            solver.profile(True)
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            solver.solve(g, phi, fpts, fgrid)
            ends[k].record(stream)
            stats.append(dict(solver.last_stats))
        torch.cuda.synchronize()
        prof = None
        if profile:
            prof = solver.profile_kernels()
            solver.profile(False)
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), stats, prof

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, stats, _ = timed(args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    value, total_ms = job_throughput(total_ms, args.steps, dist, dev)
    ms_per_step = total_ms / args.steps
    launches = int(sum(s["kernel_launches"] for s in stats))
    phi_mixed = phi.cpu().numpy().copy()

    # every kernel class timed with CUDA events around its launches (a second
    # run of the same steps, CG without graphs)
    _, pstats, kprof = timed(args.steps, profile=True)
    peak, peak_kind = measured_peaks()
    tinfo = solver.transforms_info()
    N3 = solver.N ** 3
    cg_iters_prof = sum(s["cg_iters"] for s in pstats)
    kernels = {}
    for k, (ms, n, b) in kprof.items():
        if n == 0:
            continue
        kernels[k] = {"launches_per_step": n // args.steps, "avg_launch_us": round(ms / n * 1e3, 3),
                      "ms_per_step": round(ms / args.steps, 3), "share_of_step": round(ms / args.steps / ms_per_step, 3),
                      "build_bytes_per_launch": b / n,
                      "achieved_gbs_build_bytes": round((b / n) / (ms / n * 1e-3) / 1e9, 1)}
    roofline = roofline_line(kernels, kprof, N3, cg_iters_prof, args, peak, peak_kind)

    # e2e: host buffers through kfbim_solve_host (H2D of g, f; D2H of phi)
    g_pin = torch.from_numpy(g_h).pin_memory().numpy()
    fp_pin = torch.from_numpy(fpts_h).pin_memory().numpy()
    fg_pin = torch.from_numpy(fgrid_h).pin_memory().numpy()
    phi_pin = torch.zeros(solver.n_primary, dtype=torch.float64).pin_memory().numpy()
    solver.solve_host(g_pin, phi_pin, fp_pin, fg_pin)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        solver.solve_host(g_pin, phi_pin, fp_pin, fg_pin)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": round(world * args.steps / e2e_s, 4), "unit": "solves/s",
           "h2d_bytes_per_step": int(g_pin.nbytes + fp_pin.nbytes + fg_pin.nbytes),
           "d2h_bytes_per_step": int(phi_pin.nbytes), "api": "kfbim_solve_host"}

    # FP64 comparison leg (same inputs)
    fp64 = None
    rel = None
    if not args.no_fp64:
        s64 = Solver(geom, grid, precision=FP64, **pde)
        phi64 = torch.zeros(s64.n_primary, dtype=torch.float64, device=dev)
        s64.solve(g, phi64, fpts, fgrid)
        torch.cuda.synchronize()
        reps = 2
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        ms = 0.0
        for k in range(reps):
            flush.zero_()
            ev[2 * k].record(stream)
            s64.solve(g, phi64, fpts, fgrid)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps)) / reps
        p64 = phi64.cpu().numpy()
        rel = float(np.abs(phi_mixed - p64).max() / np.abs(p64).max())
        fp64 = {"solves_per_s": round(1e3 / ms, 4), "ms_per_solve": round(ms, 2),
                "gmres_iters": s64.last_stats["gmres_iters"], "cg_iters": s64.last_stats["cg_iters"],
                "mixed_speedup": round((1e3 / ms_per_step) / (1e3 / ms), 2),
                "rel_err_vs_oracle": golden_error(args.workload, p64)}
        s64.close()

    adjoint = None
    if not args.no_adjoint and not navier:
        adjoint = adjoint_leg(solver, args, flush, stream, dev)

    batched = None
    if args.batch > 0:
        batched = batch_leg(solver, args, flush, stream, dev)

    c4 = None
    if args.batch > 0 and not navier and args.workload == "star128":
        c4 = c4_grids_leg(args, flush, stream, dev)

    large = None
    if not args.no_large and not navier:
        large = large_fp32_leg(args, flush, stream, dev, peak, peak_kind)

    cpu = None
    if rank == 0 and not args.no_cpu:
        per_solve = stats[-1]["interface_solves"]
        o = run_oracle_subprocess(args.workload, 1, per_solve)
        full = run_oracle_solve_subprocess("sphere32")
        full["all_cores"] = run_oracle_parallel("sphere32", os.cpu_count() or 1)
        cpu = {"value": round(o["value"], 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
               "value_kind": "projected",
               "sample": "projected: one oracle matvec (interface solve + trace) on %s, single thread, "
                         "%.1f s, times the %d interface solves of one GPU solve"
                         % (args.workload, o["matvec_s"], per_solve),
               "timed_solve": full, "host": host_cpu()}

    if rank == 0:
        st = stats[-1]
        desc = WORKLOAD_DESC if not navier else (
            "Navier (Lame mu=1, lambda=2) interior Dirichlet on the ellipsoid semi-axes "
            "(0.6,0.45,0.35) under a seeded rotation in [-1,1]^3, MAC grid 128^3, manufactured "
            "u_i=exp(x+y+z) sin(i+xy), GMRES tol 1e-10")
        line = {"metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64 (mixed: FP32 transforms/CG, FP64 jumps/residuals/GMRES)",
                "data": "synthetic",
                "config": {"workload": args.workload, "description": desc,
                           "precision": "mixed", "l2_flush": "512 MiB write before each step",
                           "refine_tol": solver.options.refine_tol, "inner_tol": solver.options.inner_tol,
                           "relax": solver.options.relax,
                           "n_points": solver.n_points, "n_unknowns": solver.n_primary,
                           "gmres_iters": st["gmres_iters"], "interface_solves": st["interface_solves"],
                           "cg_iters": st["cg_iters"], "refine_sweeps": st["refine_sweeps"],
                           "parallelism": "replicas" if world > 1 else "single"},
                "transforms": dict(tinfo, requested=args.transforms), "adjoint": adjoint,
                "fp32_256": large, "c4_grids": c4,
                "fp64": fp64, "rel_err_vs_fp64": rel,
                "rel_err_vs_oracle": golden_error(args.workload, phi_mixed),
                "oracle_reference": "FP64 oracle solve of the same inputs, GMRES to 1e-13 "
                                    "(tests/golden/%s_solve.npz)" % args.workload,
                "batched": batched, "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main_reference(args):
    """The oracle (single thread) on the same workload and metric: each step is
    one oracle matvec, scaled by the interface solves of one solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_solve = args.interface_solves or INTERFACE_SOLVES.get(args.workload)
    if per_solve is None:
        print(json.dumps({"impl": "reference", "unavailable": "no interface-solve count for workload %s; "
                          "pass --interface-solves" % args.workload}), flush=True)
        return
    o = run_oracle_subprocess(args.workload, args.warmup + args.steps, per_solve)
    times = o["times"][args.warmup:]
    t_mv = sum(times) / len(times)
    value = 1.0 / (t_mv * per_solve)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_mv * per_solve * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOAD_DESC},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": round(value, 6), "value_kind": "projected",
                             "sample": "projected: each step is one oracle matvec on %s (single thread), "
                                       "times %d interface solves per solve" % (args.workload, per_solve),
                             "host": host_cpu()},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.oracle_sample:
        per = a.interface_solves or INTERFACE_SOLVES.get(a.workload, 1)
        print(json.dumps(oracle_sample(a.workload, a.steps, per)))
    elif a.oracle_solve:
        print(json.dumps(oracle_full_solve(a.workload)))
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_kfbim(a)
