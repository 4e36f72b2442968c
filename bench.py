#!/usr/bin/env python3
"""Benchmark of the Ohta--Kawasaki Newton-step solver on one GB300.

Metric: FGMRES DoF x iterations per second (DoF = 2 N_v, the u and w nodal
values), mixed precision (float32 preconditioner under float64 FGMRES) as the
headline and float64 beside it, at FGMRES relative tolerance 1e-8, with
p50/p99 latency of the timesteps and of the Newton linear solves.

Workload (default): the unit square cut into 1024 x 1024 squares, each split
into two P1 triangles (1,050,625 vertices, 2,101,250 DoF); eps 0.02,
sigma 200, m 0.1, theta 0.5, dt 2e-5; u0 = m + 0.05 N(0,1) (seeded); FGMRES(30)
to 1e-8; classical Gram--Schmidt with reorthogonalisation (CGS2); six
multigrid levels (1024^2 down to a dense 33^2 coarsest solve).  A "step" is
one theta-method timestep (Newton to its stop test, every Newton step one
preconditioned FGMRES solve).  Beside the headline the JSON line carries the
float64 path, one-pass Gram--Schmidt, the nine-level hierarchy (down to 5^2),
the 3D 128^3 workload (mixed and float64) and the 3D 512^3 workload's
finest-level kernels (working set far above L2), and the oracle timed per
Newton step on the host.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ok|reference]
Under torchrun each rank runs an independent replica (the method has no
exchange step on one grid); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ok_inputs as oi  # noqa: E402

METRIC = "GMRES DoF*iter/s, mixed vs FP64 @1e-8 rel. resid; p50/p99 solve latency"
UNIT = "DoF*iter/s"
FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP64_PEAK_TFLOPS = 1.259         # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ok", "reference"], default="ok")
    ap.add_argument("--workload", default="2d_n1024", choices=sorted(oi.WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer run (short profiling runs)")
    ap.add_argument("--tuning-file", default=None,
                    help="autotuner choices: loaded from this file when it exists, saved to it at the end")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the one-pass Gram--Schmidt, nine-level and 3D runs beside the headline")
    ap.add_argument("--profile-out", default=None, help="write per-kernel samples as JSON")
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=INT",
                    help="override an integer ok_opts field of the timed runs (e.g. use_pdl=0)")
    ap.add_argument("--serving", action="store_true",
                    help="instead of the timed workload: the serving stream (Poisson arrivals) through ok_serve")
    ap.add_argument("--requests", type=int, default=256, help="serving: requests of the stream")
    ap.add_argument("--max-inflight", type=int, default=32, help="serving: requests in flight at once")
    ap.add_argument("--budget-gb", type=float, default=200.0, help="serving: device memory budget")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_across(values: dict, op: str):
    """max/sum of float scalars over ranks (identity when not distributed)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return dict(values)
    import torch
    keys = sorted(values)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(values[k]) for k in keys], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return {k: float(v) for k, v in zip(keys, t.cpu().tolist())}


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic bytes / flops per launch of the sampled kernel classes
# ---------------------------------------------------------------------------
def kernel_model(tag, wl, precision):
    """(bytes, flops, bound) per launch from the kernel contracts.

    apply_j: reads z (2 fields, float64 or float32 Z slot), the C coefficients
             (1 + NPOS float64 per vertex), writes y (2 float64); flops:
             M z1, K z2, M z2, C z1 (NOFF, 2d+1, NOFF, NOFF FMAs) + 3 per vertex.
    mg_smooth_l0: one Chebyshev step on the finest level: reads d, x, r,
             writes x, r, d' (6 values of the preconditioner type); NOFF FMAs + 4.
    cheb_mass_step: the same on M.
    """
    nv = wl.n_vertices
    d = wl.dim
    noff = 7 if d == 2 else 15
    npos = 3 if d == 2 else 7
    nax = 2 * d + 1
    bz = 4 if precision == "mixed" else 8
    bp = 4 if precision == "mixed" else 8
    if tag == "apply_j":
        by = nv * (2 * bz + 8 * (npos + 1) + 16)
        fl = nv * 2 * (noff + nax + noff + noff + 3)
        return by, fl, "alu"
    if tag in ("mg_smooth_l0", "cheb_mass_step"):
        return nv * 6 * bp, nv * 2 * (noff + 4), "hbm"
    nc = (wl.n // 2 + 1) ** d
    if tag in ("mg_tile_pre_l0", "mg_tile_post_l0"):
        # the multigrid's per-unit figure: 5 vectors per smoothing step (nu = 2
        # per launch) plus half of the level's 5 transfer/residual vectors
        # (restriction in the pre launch, prolongation in the post launch)
        return nv * 12.5 * bp, nv * 2 * (3 * noff + 12) + nc * 2 * noff, "hbm"
    if tag == "tile_mass_cstep":
        # reads v (2 float64 fields) and the C store (1 + NPOS values), writes z1 and t
        return nv * (16 + bp * (npos + 1) + bz + bp), nv * 2 * (9 * (noff + 4) + 2 * npos + 2), "hbm"
    return None, None, None


def min_bytes(tag, wl, precision):
    """Bytes a fused launch cannot avoid (its inputs and outputs once), for comparison."""
    nv, d = wl.n_vertices, wl.dim
    bp = 4 if precision == "mixed" else 8
    nc = (wl.n // 2 + 1) ** d
    if tag == "mg_tile_pre_l0":
        return nv * 2 * bp + nc * bp          # b in, x out, P^T r out
    if tag == "mg_tile_post_l0":
        return nv * 3 * bp + nc * bp          # x, b, coarse x in, x out
    return None


def launches_per_iteration(tag, opts):
    if tag == "apply_j":
        return 1
    if tag == "mg_smooth_l0":
        k = 2 if opts.get("k_R", 1) == 1 else 4
        return k * opts["n_V"] * ((opts["smooth_pre"] - 1) + (opts["smooth_post"] - 1))
    if tag == "cheb_mass_step":
        return (opts["q_A"] - 1) * (1 if opts.get("k_R", 1) == 1 else 2)
    if tag in ("mg_tile_pre_l0", "mg_tile_post_l0"):
        return 2 * opts["n_V"]
    if tag == "tile_mass_cstep":
        return 1
    return None


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1603_04570_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(tag, workload, precision):
    """DRAM bytes per launch from a committed ncu summary, if it matches these sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) == 5 and not line.startswith("#"):
            t, wk, pr, by, hs = parts
            if t == tag and wk == workload and pr == precision and hs == want:
                return float(by)
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def grid_opts(wl, precision, overrides=()):
    atol, rtol = wl.newton_tols
    o = dict(restart=wl.restart, gmres_rtol=wl.gmres_rtol, newton_atol=atol, newton_rtol=rtol,
             precision=precision, q_A=10, n_V=5, k_R=1, smooth_pre=2, smooth_post=2, use_graphs=1,
             coarse_max=32 if wl.dim == 2 else 4)
    for kv in overrides:
        k, v = kv.split("=")
        o[k] = int(v)
    return o


PROFILE_STEPS = 2


def run_precision(ok, torch, wl, precision_name, steps, warmup, rank, profile, flush, overrides=()):
    precision = ok.OK_MIXED if precision_name == "mixed" else ok.OK_FP64
    opts = grid_opts(wl, precision, overrides)
    g = ok.Grid(wl.dim, wl.n, wl.eps, wl.sigma, wl.m, wl.theta, wl.dt, **opts)
    wl_r = dataclasses.replace(wl, seed=wl.seed + rank)
    u = torch.from_numpy(oi.initial_u(wl_r)).cuda()
    w = torch.empty_like(u)
    g.init_w(u, w)
    for _ in range(warmup):
        g.timestep(u, w)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = []
    torch.cuda.synchronize()
    barrier()
    l0 = ok.ok_launch_count()
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.zero_()                          # L2 flushed before every timed step
        evs[k][0].record(stream)
        infos.append(g.timestep(u, w))
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = ok.ok_launch_count() - l0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    u_timed, w_timed = u.clone(), w.clone()    # the state after warm-up + timed steps (before sampling)
    prof = {}
    if profile:
        # per-kernel samples from separate steps: the event records they add to
        # every Arnoldi graph stay out of the timed steps above
        ok.ok_profile(g.handle, True)
        g.timestep(u, w)                       # graphs re-captured with the event nodes
        ok.ok_profile(g.handle, True)          # clear
        for _ in range(PROFILE_STEPS):
            g.timestep(u, w)
        prof = ok.ok_profile_read(g.handle)
        ok.ok_profile(g.handle, False)
    its = sum(i.gmres_its for i in infos)
    newton = sum(i.newton_its for i in infos)
    solve_lat = [i.solve_ms / max(i.newton_its, 1) for i in infos]
    res = dict(g=g, u=u, w=w, u_timed=u_timed, w_timed=w_timed, step_ms=step_ms, its=its, newton=newton, infos=infos, launches=launches,
               wall_s=t_wall, prof=prof, opts=opts, solve_lat=solve_lat)
    return res


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def e2e_run(ok, torch, res, wl, steps, flush):
    """Same metric through the C ABI with pinned host buffers (copies inside)."""
    g = res["g"]
    uh = torch.empty(g.nv, dtype=torch.float64, pin_memory=True)
    wh = torch.empty(g.nv, dtype=torch.float64, pin_memory=True)
    uh.copy_(res["u"])
    wh.copy_(res["w"])
    torch.cuda.synchronize()
    its, total = 0, 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = g.timestep(uh.numpy(), wh.numpy())
        total += time.perf_counter() - t0
        its += info.gmres_its
    nbytes = 2 * g.nv * 8
    return {"value": 2 * g.nv * its / total, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": 1e3 * total / steps,
            "api": "ok_timestep with pinned host arrays"}


def host_cpu():
    """The host's CPU model (x86 "model name"; on Arm the implementer/part codes) and core count."""
    model, part = None, None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                key = key.strip().lower()
                if key == "model name" and not model:
                    model = val.strip()
                elif key == "cpu part" and not part:
                    part = val.strip()
    except OSError:
        pass
    if not model:
        model = platform.machine() + (f" (CPU part {part})" if part else "")
    return {"cpu_model": model, "nproc": os.cpu_count()}


def cpu_baseline(wl):
    """The oracle timed per Newton step on the host (plain numpy/scipy, one
    thread: scipy's CSR products are single-threaded, the only dense work is
    the coarsest level): the 32^2 workload's five whole timesteps (FGMRES(30)
    to 1e-10) and the first Newton step of the timed workload (its FGMRES
    solve to the workload's tolerance, with the same multigrid hierarchy;
    the oracle assembles J and builds its preconditioner inside the step)."""
    from oracle.fem import Mesh, Params, System
    from oracle.solvers import Options, linear_solve, timestep
    sm = oi.SMALL_2D
    sysm = System(Mesh(sm.dim, sm.n), Params(sm.eps, sm.sigma, sm.m, sm.theta, sm.dt))
    u = oi.initial_u(sm)
    w = sysm.initial_w(u)
    atol, rtol = sm.newton_tols
    opts = Options(restart=sm.restart, gmres_rtol=sm.gmres_rtol, newton_atol=atol, newton_rtol=rtol)
    t0 = time.perf_counter()
    newton_s, its_s = 0, 0
    for _ in range(sm.steps):
        u, w, info = timestep(sysm, u, w, opts)
        newton_s += info["newton"]
        its_s += sum(info["gmres"])
    t_small = time.perf_counter() - t0
    sysm = System(Mesh(wl.dim, wl.n), Params(wl.eps, wl.sigma, wl.m, wl.theta, wl.dt))
    u0 = oi.initial_u(wl)
    w0 = sysm.initial_w(u0, solver="chebyshev")
    F = sysm.residual(u0, w0, u0, w0)
    t0 = time.perf_counter()
    _, its, rel = linear_solve(sysm, u0, -F, Options(restart=wl.restart, gmres_rtol=wl.gmres_rtol,
                                                     coarse_max=32 if wl.dim == 2 else 4))
    dt = time.perf_counter() - t0
    dof = 2 * sysm.mesh.nv
    return {"value": dof * its / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the first Newton step of {wl.name} ({dof} DoF): Jacobian assembly, preconditioner "
                      f"setup and FGMRES to {wl.gmres_rtol:g} ({its} iterations), {dt:.1f} s; "
                      f"value = DoF x iterations / that time",
            "newton_step_s": dt, "gmres_its": its, "rel_resid": rel,
            "small_2d_n32": {"timesteps": sm.steps, "newton_its": newton_s, "gmres_its": its_s,
                             "seconds": t_small, "s_per_newton_step": t_small / max(newton_s, 1)},
            **host_cpu()}


def roofline_of(res, wl, precision, total_ms):
    """Roofline of the sampled kernel class with the largest estimated share."""
    peaks, peak_kind = measured_peaks()
    best = None
    for tag, (n, tot) in res["prof"].items():
        lpi = launches_per_iteration(tag, res["opts"])
        if n == 0 or lpi is None or kernel_model(tag, wl, precision)[0] is None:
            continue
        share = tot / n * lpi * res["its"]
        if best is None or share > best[1]:
            best = (tag, share, tot / n, n)
    if not best:
        return None
    tag, share, avg_ms, n = best
    by, fl, bound = kernel_model(tag, wl, precision)
    if bound == "hbm":
        ach = by / (avg_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        unit = "GB/s"
    else:
        ach = fl / (avg_ms * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS
        unit = "TFLOP/s"
    mb = min_bytes(tag, wl, precision)
    vec_mb = wl.n_vertices * (4 if precision == "mixed" else 8) / 1e6
    # An event pair around one launch breaks the overlap that programmatic
    # dependent launch gives the chain, so a kernel inside the 2D
    # preconditioner is sampled longer than it runs: the per-kernel samples of
    # one application add up to about twice the application's own sample.
    # Scaled by that ratio, the share compares with ncu's launch list.
    share_pc = None
    pr = res["prof"]
    if tag.startswith(("mg_tile", "tile_mass", "mg_coarse")) and pr.get("precond", (0, 0))[0]:
        vc = sum(t / k for g, (k, t) in pr.items() if k and (g.startswith("mg_tile") or g == "mg_coarse"))
        parts = res["opts"]["n_V"] * 2 * vc + (pr["tile_mass_cstep"][1] / pr["tile_mass_cstep"][0]
                                                if pr.get("tile_mass_cstep", (0, 0))[0] else 0.0)
        if parts > 0:
            share_pc = share / total_ms * (pr["precond"][1] / pr["precond"][0]) / parts
    return {"kernel": tag, "bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "traffic": recorded_traffic(tag, wl.name, precision), "algorithmic_bytes_per_launch": by,
            "flops_per_launch": fl, "avg_launch_ms": avg_ms, "samples": n,
            "share_of_timed_region": share / total_ms,
            "share_scaled_to_application": share_pc,
            "fused_min_bytes_per_launch": mb,
            "frac_of_fused_min": (mb / (avg_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]) if mb else None,
            "vector_mb": vec_mb, "l2_resident": vec_mb * 4 < 129,
            "peak_source": (f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})" if bound == "hbm" else
                            "FP64 nominal: 152 SMs x 2 FMA/clk x 2.07 GHz")}


def variant(ok, torch, wl, precision_name, overrides, steps, warmup, rank, flush, ref=None, profile=False):
    """A secondary timed run (same protocol as the headline): value, iterations,
    and the relative 2-norm difference of u and w from `ref` (same steps)."""
    res = run_precision(ok, torch, wl, precision_name, steps, warmup, rank, profile, flush, overrides)
    ms = sum(res["step_ms"])
    out = {"value": wl.dofs * res["its"] / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
           "gmres_its": res["its"], "newton_its": res["newton"], "mg_levels": res["g"].levels,
           "step_p50_ms": pct(res["step_ms"], 0.5), "step_p99_ms": pct(res["step_ms"], 0.99)}
    if ref is not None:
        # same seed, warm-up and timed steps: the states after the timed steps are comparable
        for f in ("u", "w"):
            a, b = res[f + "_timed"], ref[f + "_timed"]
            out["rel_diff_" + f] = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    return out, res


def workloads_3d(ok, torch, args, rank, flush):
    """The 3D Kuhn workloads beside the 2D headline: 128^3 (mixed and float64,
    a few timesteps) and the 512^3 workload's sampled finest-level kernels
    (one timestep; its float32 vectors of 540 MB are far above the 129 MB L2,
    so these kernels stream from HBM)."""
    out = {}
    wl = oi.CUBE_128
    k = min(args.steps, 5)
    m, rm = variant(ok, torch, wl, "mixed", args.opt, k, 2, rank, flush)
    f, rf = variant(ok, torch, wl, "fp64", args.opt, k, 2, rank, flush, ref=rm)
    rm["g"].close()
    rf["g"].close()
    out[wl.name] = {"mixed": m, "fp64": f, "speedup": m["value"] / f["value"]}
    del rm, rf
    torch.cuda.empty_cache()
    wl = oi.CUBE_512
    r = run_precision(ok, torch, wl, "mixed", 1, 1, rank, True, flush, args.opt)
    ms = sum(r["step_ms"])
    out[wl.name] = {"mixed": {"value": wl.dofs * r["its"] / (ms / 1e3), "ms_per_step": ms, "steps": 1,
                              "gmres_its": r["its"], "newton_its": r["newton"], "mg_levels": r["g"].levels,
                              "tuning": [list(t) for t in r["g"].tuning()]},
                    "roofline": roofline_of(r, wl, "mixed", ms),
                    "kernel_samples": {kk: {"samples": n, "avg_ms": (t / n if n else None)}
                                       for kk, (n, t) in r["prof"].items()}}
    r["g"].close()
    del r
    torch.cuda.empty_cache()
    return out


def main_ok(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    import paper_1603_04570_gb300 as ok
    ok.load()
    if args.tuning_file and os.path.exists(args.tuning_file):
        ok.ok_tuning_load(args.tuning_file)
    wl = oi.WORKLOADS[args.workload]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    mixed = run_precision(ok, torch, wl, "mixed", args.steps, args.warmup, rank, True, flush, args.opt)
    clk = clocks.stop()
    fp64 = None if args.no_fp64 else run_precision(ok, torch, wl, "fp64", args.steps, args.warmup, rank, True,
                                                   flush, args.opt)
    e2e = None if args.no_e2e else e2e_run(ok, torch, mixed, wl, args.steps, flush)
    dof = 2 * wl.n_vertices
    total_ms = sum(mixed["step_ms"])
    agg = reduce_across({"ms": total_ms}, "max")
    units = reduce_across({"u": dof * mixed["its"]}, "sum")["u"]
    value = units / (agg["ms"] / 1e3)
    roof = roofline_of(mixed, wl, "mixed", total_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": agg["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32 (mixed)", "data": "synthetic",
        "config": {"workload": wl.name, "dim": wl.dim, "n": wl.n, "vertices": wl.n_vertices, "dofs": dof,
                   "eps": wl.eps, "sigma": wl.sigma, "m": wl.m, "theta": wl.theta, "dt": wl.dt,
                   "restart": wl.restart, "gmres_rtol": wl.gmres_rtol, "mg_levels": mixed["g"].levels,
                   "gram_schmidt": {0: "DGKS-conditional second pass", 1: "CGS2 (classical, reorthogonalised)",
                                    2: "one classical pass"}[mixed["g"].opts.reorth],
                   "precision": "mixed (float32 preconditioner, float64 FGMRES/J/residual)",
                   "l2": "flushed by a 512 MB write before every timed step", "parallelism": f"replicas x{world}",
                   **({"overrides": args.opt} if args.opt else {})},
        "gmres_its": mixed["its"], "newton_its": mixed["newton"],
        "its_per_newton": mixed["its"] / max(mixed["newton"], 1),
        "latency": {"step_p50_ms": pct(mixed["step_ms"], 0.5), "step_p99_ms": pct(mixed["step_ms"], 0.99),
                    "newton_solve_p50_ms": pct(mixed["solve_lat"], 0.5),
                    "newton_solve_p99_ms": pct(mixed["solve_lat"], 0.99)},
        "roofline": roof, "e2e": e2e, "gpu_launches": mixed["launches"], "clocks": clk,
        "tuning": [list(t) for t in mixed["g"].tuning()],
        "kernel_samples": {k: {"samples": n, "avg_ms": (t / n if n else None)} for k, (n, t) in mixed["prof"].items()},
    }
    if fp64 is not None:
        fms = sum(fp64["step_ms"])
        du = float(torch.linalg.norm(mixed["u_timed"] - fp64["u_timed"]) / torch.linalg.norm(fp64["u_timed"]))
        dw = float(torch.linalg.norm(mixed["w_timed"] - fp64["w_timed"]) / torch.linalg.norm(fp64["w_timed"]))
        out["fp64"] = {"value": dof * fp64["its"] / (fms / 1e3), "ms_per_step": fms / args.steps,
                       "gmres_its": fp64["its"], "newton_its": fp64["newton"],
                       "step_p50_ms": pct(fp64["step_ms"], 0.5), "step_p99_ms": pct(fp64["step_ms"], 0.99),
                       "kernel_samples": {k: {"samples": n, "avg_ms": (t / n if n else None)}
                                          for k, (n, t) in fp64["prof"].items()}}
        out["mixed_vs_fp64"] = {"speedup": out["value"] / out["fp64"]["value"], "rel_diff_u": du,
                                "rel_diff_w": dw}
    if not args.no_variants:
        ref = fp64 if fp64 is not None else None
        v1, r1 = variant(ok, torch, wl, "mixed", list(args.opt) + ["reorth=2"], args.steps, args.warmup, rank,
                         flush, ref=ref)
        r1["g"].close()
        v1["what"] = "one classical Gram-Schmidt pass per Arnoldi step (no reorthogonalisation)"
        out["one_pass_gram_schmidt"] = v1
        if wl.dim == 2:
            v2, r2 = variant(ok, torch, wl, "mixed", list(args.opt) + ["coarse_max=4"], args.steps, args.warmup,
                             rank, flush, ref=ref)
            r2["g"].close()
            v2["what"] = "nine multigrid levels (1024^2 down to a dense 5^2 coarsest solve)"
            out["mg_9_levels"] = v2
            del r1, r2
        if wl.name == "2d_n1024":
            out["workloads"] = workloads_3d(ok, torch, args, rank, flush)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if args.tuning_file:
        ok.ok_tuning_save(args.tuning_file)
    if args.profile_out and rank == 0:
        json.dump(out, open(args.profile_out, "w"), indent=1, default=str)
    if rank == 0:
        print(json.dumps(out, default=lambda o: None))
    mixed["g"].close()
    if fp64 is not None:
        fp64["g"].close()


def main_reference(args):
    """The oracle (plain numpy/scipy, host cores) on the same workload and metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle.fem import Mesh, Params, System
    from oracle.solvers import Preconditioner, fgmres
    wl = oi.WORKLOADS[args.workload]
    sysm = System(Mesh(wl.dim, wl.n), Params(wl.eps, wl.sigma, wl.m, wl.theta, wl.dt))
    u0 = oi.initial_u(wl)
    w0 = sysm.initial_w(u0, solver="chebyshev")
    F = sysm.residual(u0, w0, u0, w0)
    J = sysm.jacobian(u0)
    P = Preconditioner(sysm, u0, mode="inexact", q_A=10, n_V=5, k_R=1, coarse_max=32 if wl.dim == 2 else 4)
    per_step = 2
    run = lambda: fgmres(lambda z: J @ z, P.apply, -F, restart=wl.restart, rtol=wl.gmres_rtol, max_its=per_step)[1]
    for _ in range(args.warmup):
        run()
    times, its = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        its += run()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    dof = 2 * sysm.mesh.nv
    value = dof * its / total
    sample = (f"each step: {per_step} FGMRES iterations of the first Newton solve of {wl.name} "
              f"({dof} DoF), oracle scipy CSR operators, 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "dim": wl.dim, "n": wl.n, "dofs": dof, "restart": wl.restart,
                   "gmres_rtol": wl.gmres_rtol},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1, "sample": sample,
                         **host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def serve_stream(ok, torch, stream, prec, args):
    """One pass of the serving stream through ok_serve at one precision."""
    reqs = []
    for arrival, wl in stream:
        atol, rtol = wl.newton_tols
        u = torch.from_numpy(oi.initial_u(wl)).cuda()
        reqs.append(dict(dim=wl.dim, n=wl.n, eps=wl.eps, sigma=wl.sigma, m=wl.m, theta=wl.theta, dt=wl.dt,
                         u=u, w=torch.zeros_like(u), steps=wl.steps, init_w=True, arrival=arrival,
                         opts=dict(precision=prec, restart=wl.restart, gmres_rtol=wl.gmres_rtol,
                                   newton_atol=atol, newton_rtol=rtol,
                                   coarse_max=32 if (wl.dim == 2 and wl.n >= 128) else 4)))
    torch.cuda.synchronize()
    st, res, info = ok.ok_serve(reqs, args.max_inflight, int(args.budget_gb * (1 << 30)))
    lat = [r.t_done - a for r, (a, _) in zip(res, stream)]
    wait = [r.t_admit - a for r, (a, _) in zip(res, stream)]
    units = sum(2 * wl.n_vertices * r.gmres_its for r, (_, wl) in zip(res, stream))
    return {
        "p50_ms": pct(lat, 0.5) * 1e3, "p99_ms": pct(lat, 0.99) * 1e3,
        "admission_wait_p50_ms": pct(wait, 0.5) * 1e3, "admission_wait_p99_ms": pct(wait, 0.99) * 1e3,
        "requests": len(stream), "completed": info.completed, "failed": info.failed, "status": st,
        "seconds": info.seconds, "throughput_req_s": info.completed / info.seconds,
        "dof_iter_per_s": units / info.seconds, "peak_inflight": info.peak_inflight,
        "peak_cohort": info.peak_cohort, "cohort_timesteps": info.cohort_steps,
        "errors": sorted({r.message.decode() for r in res if r.status != 0}),
        "peak_estimated_gb": info.peak_bytes / 2 ** 30,
    }, [(q["u"], q["w"]) for q in reqs]


def main_serving(args):
    """The serving stream: whole simulations with Poisson arrivals, admitted by
    ok_serve (continuous batching: same-grid requests advance as cohorts with
    shared launches); latency = completion - arrival per request; mixed
    precision, then float64 on the same stream, with their difference."""
    import torch
    import paper_1603_04570_gb300 as ok
    ok.load()
    stream = oi.serving_requests(args.requests)
    clocks = ClockSampler(0)
    clocks.start()
    mixed, sm = serve_stream(ok, torch, stream, ok.OK_MIXED, args)
    clk = clocks.stop()
    fp64, sf = (None, None) if args.no_fp64 else serve_stream(ok, torch, stream, ok.OK_FP64, args)
    out = {
        "metric": "serving latency p50/p99 (completion - arrival) of whole simulations", "impl": "ok",
        "value": mixed["p99_ms"], "unit": "ms (p99)", "higher_is_better": False, "n_gpus": 1,
        **mixed, "precision": "mixed",
        "config": {"workload": "serving stream: Poisson arrivals at 40 req/s; 2D {64..512}^2 and 3D {32..96}^3, "
                               "5-50 timesteps each", "max_inflight": args.max_inflight,
                   "budget_gb": args.budget_gb},
        "data": "synthetic", "clocks": clk,
    }
    if fp64 is not None:
        diff = max(float(torch.linalg.norm(a[0] - b[0]) / torch.linalg.norm(b[0])) for a, b in zip(sm, sf))
        out["fp64"] = fp64
        out["mixed_vs_fp64_max_rel_diff_u"] = diff
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.serving:
        main_serving(a)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ok(a)
