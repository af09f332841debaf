"""Benchmark: DOF-stage updates per second of the Boltzmann-BGK SSP-RK3 hot path on GB300.

One "step" is one SSP-RK3 step (three stages) over the whole Taylor-Green workload: 16^3 hexahedra
at p = 3 (262,144 points) x 24^3 velocities (13,824) = 3.62e9 degrees of freedom; each stage
advects every velocity, relaxes towards the conservative Maxwellian and recomputes moments and the
Newton solve. value = n_x * N_v * 3 / (seconds per step), timed over K steps of the captured CUDA graph;
a second pass of K steps launched directly, with CUDA events around every launch, gives the roofline's
per-launch durations. f (14.5 GB per array) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torchrun) runs N independent replicas, one per GPU, with no data-path collective
(the single periodic domain is not partitioned); value is the sum over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
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

from paper_2308_06196_gb300 import workloads as W  # noqa: E402

METRIC = "DOF-stage updates/sec (x-pts x v-pts) & %HBM roofline, FP32/FP64-split vs all-FP64"
UNIT = "DOF-stage/s"
WORKLOAD = "taylor_green"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def stage_traffic():
    """DRAM bytes per stage launch from the committed ncu summary, if it was taken on this source."""
    p = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != stage_source_sha():
        return None
    return d.get("dram_bytes_per_launch")


NOMINAL_HBM_GBS = 7900.0  # GB300's nominal HBM3e bandwidth, for context beside the measured copy peak


def stage_source_sha():
    """Hash of the sources of the hexahedral stage kernel (the counters are void once they change)."""
    h = hashlib.sha256()
    for fn in ("k_stage3s.cuh", "stage_common.cuh", "bgk_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2308_06196_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()


def cpu_sample_problem():
    """Bounded sample of the Taylor-Green workload for the CPU oracle: an 8 x 4 x 4-element periodic
    box of the same mesh spacing at p = 3 with the full 24^3 velocity grid (128 elements, 1.1e8 DOF;
    about 4 s per RK step on 16 cores)."""
    c = W.config(WORKLOAD)
    h = (c["hi"][0] - c["lo"][0]) / c["nelem"][0]
    ne = (8, 4, 4)
    return dict(c, nelem=ne, hi=tuple(c["lo"][d] + ne[d] * h for d in range(3)))


def run_oracle(steps: int, warmup: int):
    from oracle import oracle as orc

    c = cpu_sample_problem()
    k = W.mesh_kwargs(c)
    pr = orc.Problem(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
    pr.set_state(W.prim_field(WORKLOAD, pr.points()))
    dt = pr.dt(c["cfl"])
    pr.step(dt, warmup)
    t0 = time.perf_counter()
    pr.step(dt, steps)
    sec = time.perf_counter() - t0
    dof = pr.npts * pr.nvel
    cores = os.cpu_count()
    return dof * 3 * steps / sec, sec / steps, cores, dof, c


def bench_batch(steps: int, warmup: int, stream, torch, members: int = 0) -> dict:
    """The ensemble of independent 1-D Sod tubes (uneven mesh, degree and velocity grid) in one batch:
    one persistent stage launch and one Newton launch per RK stage, the step under a CUDA graph, tile
    lengths from the batch autotuner; then the same members stepped one after another through their
    own graphs, for the batching gain."""
    from paper_2308_06196_gb300.bgk import Batch, Solver

    cb = W.config("sod_ensemble")
    if members:
        cb["members"] = members
    members = W.sod_members(**cb)
    sol = []
    for m in members:
        k = W.mesh_kwargs(m)
        s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                   bc=m["bc"], bc_state=m["bc_state"], chunks=1)
        s.set_stream(stream.cuda_stream)
        s.set_state(W.prim_sod(s.points(), m["left"], m["right"]))
        sol.append(s)
    dts = [s.dt(cb["cfl"]) for s in sol]
    b = Batch(sol)
    b.set_stream(stream.cuda_stream)
    b.autotune()
    dof = sum(s.ndof for s in sol)
    b.step(dts, warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(dts, steps)
    e1.record(stream)
    b.synchronize()
    ms = e0.elapsed_time(e1) / steps
    b.set_timing(True)
    b.step(dts, steps)
    tm = b.timing()
    b.set_timing(False)
    b.synchronize()
    # the members alone, one after another (each through its own captured graph)
    for s, dt in zip(sol, dts):
        s.step(dt, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for s, dt in zip(sol, dts):
        s.step(dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_alone = e0.elapsed_time(e1) / steps
    stage_avg = tm["stage_ms"] / max(1, tm["stage_launches"])
    out = {"workload": "sod_ensemble", "members": len(sol), "dof": dof, "tasks": b.tasks,
           "value": dof * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "stage_avg_ms": stage_avg, "stage_achieved_gbs": tm["stage_alg_bytes"] / (stage_avg * 1e-3) / 1e9,
           "newton_avg_ms": tm["newton_ms"] / max(1, tm["newton_launches"]),
           "launches_per_step": (tm["stage_launches"] + tm["newton_launches"]) / steps,
           "members_alone_ms_per_step": ms_alone, "batching_speedup": ms_alone / ms}
    b.close()
    for s in sol:
        s.close()
    return out


def max_over_ranks(values, dist, device):
    """Each timing's maximum over all ranks: the slowest replica sets the job's time."""
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_value(dof_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job DOF-stage updates per second: every rank steps its own replica of the workload."""
    return dof_per_rank * 3 * world / (ms_per_step * 1e-3)


def timed_steps(s, dt, steps, warmup, stream, torch):
    """ms per step through the graph, and the stage timing of the same number of steps."""
    s.step(dt, warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(dt, steps)
    e1.record(stream)
    s.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.set_timing(True)
    s.step(dt, steps)
    tm = s.timing()
    s.set_timing(False)
    s.synchronize()
    stage_avg = tm["stage_ms"] / max(1, tm["stage_launches"])
    return ms, {"stage_avg_ms": stage_avg, "stage_achieved_gbs": tm["stage_alg_bytes"] / (stage_avg * 1e-3) / 1e9,
                "newton_avg_ms": tm["newton_ms"] / max(1, tm["newton_launches"])}


def bench_mach5(steps: int, warmup: int, stream, torch, yz_elements: int = 0) -> dict:
    """The Mach-5 duct at full size in the FP32-split form (positivity limiter on, general kernel),
    then the plain all-FP64 form on the one-element-wide duct of the same x-mesh for the same steps:
    the flow is y/z-homogeneous, so the two must agree; their moments' largest scaled difference."""
    from paper_2308_06196_gb300.bgk import FP64, Solver

    c = W.config("mach5")
    if yz_elements:  # a narrower duct of the same element size (profiling)
        ne = c["nelem"]
        c = dict(c, nelem=(ne[0], yz_elements, yz_elements),
                 hi=(c["hi"][0], c["hi"][1] * yz_elements / ne[1], c["hi"][2] * yz_elements / ne[2]))
    bc, bcs = W.mach5_bc(c)
    k = W.mesh_kwargs(c)
    s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"], bc=bc,
               bc_state=bcs, limiter=c["limiter"])
    s.set_stream(stream.cuda_stream)
    prim = W.prim_mach5(s.points(), c)
    s.set_state(prim)
    g = s.autotune()
    dt = s.dt(c["cfl"])
    ms, st = timed_steps(s, dt, steps, warmup, stream, torch)
    total = warmup + 2 * steps
    Q = s.moments()
    dof, npts = s.ndof, s.npts
    s.close()
    ne, n1 = c["nelem"], c["p"] + 1
    Qx = Q.reshape(ne[2], ne[1], ne[0], n1, n1, n1, 5).transpose(2, 5, 0, 1, 3, 4, 6).reshape(ne[0], n1, -1, 5)
    hy = (c["hi"][1] - c["lo"][1]) / ne[1]
    c64 = dict(c, nelem=(ne[0], 1, 1), hi=(c["hi"][0], hy, hy))
    k64 = W.mesh_kwargs(c64)
    s64 = Solver(k64["dim"], k64["nelem"], k64["lo"], k64["hi"], k64["p"], k64["nv"], k64["vlo"], k64["vhi"],
                 k64["tau"], bc=bc, bc_state=bcs, limiter=c["limiter"], precision=FP64)
    s64.set_stream(stream.cuda_stream)
    s64.set_state(W.prim_mach5(s64.points(), c64))
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s64.step(dt, 1)
    torch.cuda.synchronize()
    h0.record(stream)
    s64.step(dt, total - 1)
    h1.record(stream)
    Q64 = s64.moments().reshape(ne[0], n1, n1, n1, 5)[:, 0, 0, :, :]
    ms64 = h0.elapsed_time(h1) / (total - 1)
    dof64 = s64.ndof
    s64.close()
    rho = Q64[..., 0]
    th = (2.0 / 3.0) * (Q64[..., 4] / rho - 0.5 * (Q64[..., 1:4] ** 2).sum(-1) / rho**2)
    scale = np.array([rho.max()] + [(rho * np.sqrt(th)).max()] * 3 + [Q64[..., 4].max()])
    homog = float(np.abs(Qx - Qx[:, :, :1]).max())
    err = float((np.abs(Qx[:, :, 0, :] - Q64) / scale).max())
    # the plain FP64 form on a 2 x 2-element-wide duct too (y/z-homogeneous: every y/z column equals the
    # one-element-wide duct's up to the FP64 form's round-off in the vanishing y/z derivatives)
    c2 = dict(c, nelem=(ne[0], 2, 2), hi=(c["hi"][0], 2 * hy, 2 * hy))
    k2 = W.mesh_kwargs(c2)
    s2 = Solver(k2["dim"], k2["nelem"], k2["lo"], k2["hi"], k2["p"], k2["nv"], k2["vlo"], k2["vhi"], k2["tau"],
                bc=bc, bc_state=bcs, limiter=c["limiter"], precision=FP64)
    s2.set_stream(stream.cuda_stream)
    s2.set_state(W.prim_mach5(s2.points(), c2))
    s2.step(dt, total)
    Q2 = s2.moments().reshape(2, 2, ne[0], n1, n1, n1, 5).transpose(2, 5, 0, 1, 3, 4, 6).reshape(ne[0], n1, -1, 5)
    s2.close()
    err2 = float((np.abs(Q2 - Q64[:, :, None, :]) / scale).max())
    return {"workload": "mach5", "dof": dof, "n_x": npts, "value": dof * 3 / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, **st, "tiles_per_task": g, "limiter": True, "steps_compared": total,
            "yz_homogeneity_max_abs_diff": homog,
            "fp64_narrow_duct": {"dof": dof64, "value": dof64 * 3 / (ms64 * 1e-3), "unit": UNIT,
                                 "ms_per_step": ms64, "moments_max_rel_diff_fp32_split": err,
                                 "duct_2x2_moments_max_rel_diff": err2}}


def bench_planar(steps: int, warmup: int, stream, torch) -> dict:
    """The transverse shear wave in the two-dimensional velocity space (m = 2) on a 65,536-element
    periodic line in the FP32-split form, then the plain all-FP64 form for the same steps from the same
    state: ms per step, the stage kernel's achieved bandwidth, and the two forms' largest scaled
    moment difference."""
    from paper_2308_06196_gb300.bgk import FP64, Solver

    c = W.config("planar_shear")
    k = W.mesh_kwargs(c)
    out = {"workload": "planar_shear", "mesh": f"{c['nelem'][0]} line elements p={c['p']}, periodic",
           "nv": list(c["nv"]), "velocity_dimension": 2}
    Q = {}
    for name, prec in (("fp32_split", 0), ("fp64", FP64)):
        s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                   precision=prec)
        s.set_stream(stream.cuda_stream)
        s.set_state(W.prim_shear(s.points(), c["amp"]))
        if prec == 0:
            out["tiles_per_task"] = s.autotune()
            dt = s.dt(c["cfl"])
            ms, st = timed_steps(s, dt, steps, warmup, stream, torch)
            n_total = warmup + 2 * steps
            out.update({"dof": s.ndof, "value": s.ndof * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, **st})
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.step(dt, 1)
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(dt, n_total - 1)
            e1.record(stream)
            s.synchronize()
            ms64 = e0.elapsed_time(e1) / (n_total - 1)
            out["fp64"] = {"value": s.ndof * 3 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64}
        Q[name] = s.moments()
        s.close()
    q32, q64 = Q["fp32_split"], Q["fp64"]
    scale = np.array([np.abs(q64[:, 0]).max()] + [np.abs(q64[:, 0]).max()] * 3 + [np.abs(q64[:, 4]).max()])
    out["steps_compared"] = n_total
    out["moments_max_rel_diff_fp32_split"] = float((np.abs(q32 - q64).max(axis=0) / scale).max())
    out["fp64"]["speedup_of_fp32_split"] = out["value"] / out["fp64"]["value"]
    return out


def bench_channel(steps: int, warmup: int, stream, torch) -> dict:
    """The rarefied channel at full size (32 x 16 x 4 hexahedra at p = 2, 32^3 velocities, diffuse
    isothermal walls in y, body force 0.01 in x, Kn = 0.1) in the FP32-split form (general kernel: wall
    ghosts with their per-point densities, the force source), then the plain all-FP64 form for the same
    steps from the same state: ms per step, the stage kernel's achieved bandwidth and the two forms'
    largest scaled moment difference."""
    from paper_2308_06196_gb300.bgk import FP64, Solver

    c = W.config("channel")
    k = W.mesh_kwargs(c)
    out = {"workload": "channel", "mesh": "32x16x4 hex p=2 on [0,2]x[0,1]x[0,0.25], diffuse walls in y",
           "nv": list(c["nv"]), "tau": c["tau"], "force": list(c["force"])}
    Q = {}
    for name, prec in (("fp32_split", 0), ("fp64", FP64)):
        s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                   bc=c["bc"], bc_state=c["bc_state"], body_force=c["force"], precision=prec)
        s.set_stream(stream.cuda_stream)
        s.set_state(W.prim_field("channel", s.points()))
        if prec == 0:
            out["tiles_per_task"] = s.autotune()
            dt = s.dt(c["cfl"])
            ms, st = timed_steps(s, dt, steps, warmup, stream, torch)
            n_total = warmup + 2 * steps
            out.update({"dof": s.ndof, "dt": dt, "value": s.ndof * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                        **st})
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.step(dt, 1)
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(dt, n_total - 1)
            e1.record(stream)
            s.synchronize()
            ms64 = e0.elapsed_time(e1) / (n_total - 1)
            out["fp64"] = {"value": s.ndof * 3 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64}
        Q[name] = s.moments()
        s.close()
    q32, q64 = Q["fp32_split"], Q["fp64"]
    rho = q64[:, 0]
    th = (2.0 / 3.0) * (q64[:, 4] / rho - 0.5 * (q64[:, 1:4] ** 2).sum(-1) / rho**2)
    scale = np.array([rho.max()] + [(rho * np.sqrt(th)).max()] * 3 + [q64[:, 4].max()])
    out["steps_compared"] = n_total
    out["moments_max_rel_diff_fp32_split"] = float((np.abs(q32 - q64).max(axis=0) / scale).max())
    out["fp64"]["speedup_of_fp32_split"] = out["value"] / out["fp64"]["value"]
    return out


def bench_quad(steps: int, warmup: int, stream, torch, elements: int = 0) -> dict:
    """The planar Taylor-Green vortex on quadrilaterals (dim = 2) in the two-dimensional velocity space,
    FP32-split form: ms per step and the quadrilateral stage kernel's achieved bandwidth."""
    from paper_2308_06196_gb300.bgk import Solver

    c = W.config("planar_tg")
    if elements:  # fewer, larger elements on the same box (profiling)
        c = W.config("planar_tg", nelem=(elements, elements))
    k = W.mesh_kwargs(c)
    s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
    s.set_stream(stream.cuda_stream)
    s.set_state(W.prim_planar_tg(s.points(), c["mach"]))
    g = s.autotune()
    dt = s.dt(c["cfl"])
    ms, st = timed_steps(s, dt, steps, warmup, stream, torch)
    out = {"workload": "planar_tg", "mesh": f"{c['nelem'][0]}^2 quadrilaterals p=3 on [0,2pi]^2", "nv": list(c["nv"]),
           "dof": s.ndof, "value": s.ndof * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "dt": dt,
           "tiles_per_task": g, **st}
    s.close()
    return out


def bench_curved(steps: int, warmup: int, stream, torch, elements: int = 0) -> dict:
    """The Taylor-Green workload on curvilinear hexahedra: the box's solution nodes displaced by the
    smooth periodic sine mapping (amplitude 0.3 element widths), metric terms from bgk_set_geometry,
    the curvilinear stage kernel (per-lane upwinding, reference-space flux)."""
    from paper_2308_06196_gb300.bgk import Solver

    c = W.config(WORKLOAD)
    if elements:  # fewer, larger elements on the same box (profiling)
        c = W.config(WORKLOAD, nelem=(elements,) * 3)
    k = W.mesh_kwargs(c)
    s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
    s.set_stream(stream.cuda_stream)
    X = W.curved_nodes(s.points(), c["lo"], c["hi"], c["nelem"], 0.3, kind="sine")
    s.set_geometry(X)
    s.set_state(W.prim_field(WORKLOAD, X))
    g = s.autotune()
    dt = s.dt(c["cfl"])
    ms, st = timed_steps(s, dt, steps, warmup, stream, torch)
    out = {"workload": "taylor_green on curvilinear hexahedra (sine mapping, 0.3 h)", "dof": s.ndof,
           "value": s.ndof * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "dt": dt, "tiles_per_task": g, **st}
    Q = s.moments()
    s.close()
    # the plain all-FP64 form on the same curved mesh for the same steps from the same state: its time
    # and the largest scaled moment difference (full-size parity of the curvilinear kernel)
    from paper_2308_06196_gb300.bgk import FP64

    n_total = warmup + 2 * steps
    s64 = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"], precision=FP64)
    s64.set_stream(stream.cuda_stream)
    s64.set_geometry(X)
    s64.set_state(W.prim_field(WORKLOAD, X))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s64.step(dt, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    s64.step(dt, n_total - 1)
    e1.record(stream)
    Q64 = s64.moments()
    ms64 = e0.elapsed_time(e1) / (n_total - 1)
    s64.close()
    rho = Q64[:, 0]
    th = (2.0 / 3.0) * (Q64[:, 4] / rho - 0.5 * (Q64[:, 1:4] ** 2).sum(1) / rho**2)
    scale = np.array([rho.max()] + [(rho * np.sqrt(th)).max()] * 3 + [np.abs(Q64[:, 4]).max()])
    out["fp64"] = {"value": out["dof"] * 3 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                   "steps_compared": n_total,
                   "moments_max_rel_diff_fp32_split": float((np.abs(Q - Q64).max(axis=0) / scale).max())}
    # the same mesh as an unstructured one (table-driven neighbours): every element's local axes rotated
    # at random, in the grid's own element order (as a locality-ordered mesh) and in a random order (no
    # locality at all); the same steps must give the same moments up to FP32 rounding
    for name, shuffle in (("unstructured", False), ("unstructured_random_order", True)):
        u = W.unstructured_box(c["nelem"], c["p"], seed=0, shuffle=shuffle)
        m = u["node_map"]
        s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
        s.set_stream(stream.cuda_stream)
        s.set_connectivity(u["nbr"], u["nface"], u["orient"])
        s.set_geometry(X[m])
        s.set_state(W.prim_field(WORKLOAD, X[m]))
        s.autotune()
        ms_u, st_u = timed_steps(s, dt, steps, warmup, stream, torch)
        Qu = s.moments()
        s.close()
        out[name] = {"value": s.ndof * 3 / (ms_u * 1e-3), "unit": UNIT, "ms_per_step": ms_u, **st_u,
                     "moments_max_rel_diff_vs_structured": float(np.abs(Qu - Q[m]).max() / np.abs(Q).max())}
    return out


def bench_variants(steps: int, warmup: int, stream, torch, k: dict, prim_dev, dt: float) -> dict:
    """The Taylor-Green workload with the widened rows switched on one at a time: the positivity
    limiter and the variable collision time (both in the general hexahedral kernel), and the
    continuous-Maxwellian ablation (no Newton solve)."""
    from paper_2308_06196_gb300.bgk import MAXWELLIAN_CONTINUOUS, Solver

    out = {}
    for name, opts in (("limiter", dict(limiter=True)),
                       ("variable_tau", dict(mu_ref=1e-3, mu_omega=0.81)),
                       ("continuous_maxwellian", dict(maxwellian=MAXWELLIAN_CONTINUOUS))):
        s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"], **opts)
        s.set_stream(stream.cuda_stream)
        s.set_state(prim_dev)
        s.autotune()
        ms, st = timed_steps(s, min(dt, s.dt(0.1)), steps, warmup, stream, torch)
        out[name] = {"value": s.ndof * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, **st}
        s.close()
    return out


def bench_ablation() -> dict:
    """The paper's central claim (Sec. 2.1, Eq. 13 and the text after it), measured: the drift of the
    total mass and energy of a periodic 3-D box after 20 steps with the discretely-conservative
    Maxwellian and with the sampled continuous one, for velocity grids of 8^3, 12^3 and 16^3."""
    from paper_2308_06196_gb300.bgk import MAXWELLIAN_CONTINUOUS, MAXWELLIAN_CONSERVATIVE, Solver

    # the discrete spatial integral: tensor Gauss-Legendre weights of the p = 2 nodes (x fastest)
    w = np.polynomial.legendre.leggauss(3)[1]
    Wn = np.einsum("i,j,k->kji", w, w, w).ravel()

    def total(Q):
        return (Q.reshape(-1, Wn.size, 5) * Wn[None, :, None]).sum((0, 1))

    out = {}
    for N in (8, 12, 16):
        row = {}
        for name, mode in (("conservative", MAXWELLIAN_CONSERVATIVE), ("continuous", MAXWELLIAN_CONTINUOUS)):
            s = Solver(3, [4, 4, 4], [0.0] * 3, [1.0] * 3, 2, (N, N, N), (-5.0,) * 3, (5.0,) * 3, 5e-3,
                       maxwellian=mode)
            s.set_state(W.smooth_prim(s.points(), 3, seed=1, amp=0.3))
            Q0 = total(s.moments())
            s.step(s.dt(0.1), 20)
            d = np.abs(total(s.moments()) - Q0)
            row[name] = float(max(d[0] / abs(Q0[0]), d[4] / abs(Q0[4])))
            s.close()
        out[f"N{N}"] = row
    return {"workload": "periodic box 4^3 hex p=2, tau=5e-3, 20 steps", "metric": "max relative drift of total "
            "mass and energy", **out}


def moment_scales(Q):
    """Component scales of the moment distance: rho for mass, rho sqrt(theta) for momentum (a component
    of the mean velocity can vanish identically), E for energy; theta with the velocity dimension 3."""
    rho = Q[:, 0]
    th = (2.0 / 3.0) * (Q[:, 4] / rho - 0.5 * (Q[:, 1:4] ** 2).sum(1) / rho**2)
    return np.array([rho.max()] + [(rho * np.sqrt(th)).max()] * 3 + [np.abs(Q[:, 4]).max()])


def pair_accuracy(make, prim_fn, steps: int, dt_cfl: float, stream, torch) -> dict:
    """One workload in the FP32-split and the all-FP64 form from the same state for the same steps:
    both forms' ms per step, and the FP32-split form's distance from the FP64 one in the moments
    (largest scaled component difference) and in f (max |f32 - f64| / max |f64|, on the device)."""
    from paper_2308_06196_gb300.bgk import FP64

    out = {}
    sol = {}
    for name, prec in (("fp32_split", 0), ("fp64", FP64)):
        s = make(prec)
        s.set_stream(stream.cuda_stream)
        s.set_state(prim_fn(s.points()))
        if prec == 0:
            s.autotune()
        dt = s.dt(dt_cfl) if name == "fp32_split" else out["dt"]
        out["dt"] = dt
        s.step(dt, 1)  # graph capture, timed with the rest below as part of the run
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(dt, steps - 1)
        e1.record(stream)
        s.synchronize()
        out[f"{name}_ms_per_step"] = e0.elapsed_time(e1) / max(1, steps - 1)
        sol[name] = s
    Q32, Q64 = sol["fp32_split"].moments(), sol["fp64"].moments()
    df, fm = sol["fp32_split"].f_distance(sol["fp64"])
    out.update({"dof": sol["fp64"].ndof, "steps": steps,
                "moments_max_rel_diff": float((np.abs(Q32 - Q64).max(axis=0) / moment_scales(Q64)).max()),
                "f_max_abs_diff_rel": df / fm,
                "speedup_of_fp32_split": out["fp64_ms_per_step"] / out["fp32_split_ms_per_step"]})
    for s in sol.values():
        s.close()
    return out


def bench_accuracy(steps: int, stream, torch, sod_oracle_members: int = 3) -> dict:
    """The FP32-split form's accuracy after `steps` RK steps, per workload, against the all-FP64 GPU form
    (and, for the line workloads, the FP64 CPU oracle), with the time per step of both forms:
    the Taylor-Green box and the channel at full size; the Mach-5 duct on its one-element-wide form
    (y/z-homogeneous, so it stands for the full duct, whose own moments are compared with the FP64 duct
    too); the Sod ensemble as one FP32-split batch against its members one after another in the FP64 form,
    and a few members against the oracle; the 1-D periodic workload against the oracle."""
    from paper_2308_06196_gb300.bgk import FP64, Batch, Solver

    res = {"steps": steps, "tolerance_moments": 1e-5}
    c = W.config("taylor_green")
    k = W.mesh_kwargs(c)
    res["taylor_green"] = pair_accuracy(
        lambda prec: Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                            precision=prec), lambda x: W.prim_field("taylor_green", x), steps, c["cfl"], stream, torch)
    c = W.config("channel")
    k = W.mesh_kwargs(c)
    res["channel"] = pair_accuracy(
        lambda prec: Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                            bc=c["bc"], bc_state=c["bc_state"], body_force=c["force"], precision=prec),
        lambda x: W.prim_field("channel", x), steps, c["cfl"], stream, torch)
    # Mach 5: the one-element-wide duct in both forms, then the full duct (FP32-split) against it
    c = W.config("mach5")
    bc, bcs = W.mach5_bc(c)
    ne = c["nelem"]
    hy = (c["hi"][1] - c["lo"][1]) / ne[1]
    cn = dict(c, nelem=(ne[0], 1, 1), hi=(c["hi"][0], hy, hy))
    kn = W.mesh_kwargs(cn)
    m5 = pair_accuracy(
        lambda prec: Solver(kn["dim"], kn["nelem"], kn["lo"], kn["hi"], kn["p"], kn["nv"], kn["vlo"], kn["vhi"],
                            kn["tau"], bc=bc, bc_state=bcs, limiter=True, precision=prec),
        lambda x: W.prim_mach5(x, cn), steps, c["cfl"], stream, torch)
    m5["mesh"] = f"{ne[0]}x1x1 hex p=2 (the duct's y/z-homogeneous form)"
    k = W.mesh_kwargs(c)
    s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"], bc=bc,
               bc_state=bcs, limiter=True)
    s.set_stream(stream.cuda_stream)
    s.set_state(W.prim_mach5(s.points(), c))
    s.autotune()
    s.step(m5["dt"], steps)
    Q = s.moments()
    s.close()
    n1 = c["p"] + 1
    Qx = Q.reshape(ne[2], ne[1], ne[0], n1, n1, n1, 5).transpose(2, 5, 0, 1, 3, 4, 6).reshape(ne[0], n1, -1, 5)
    s64 = Solver(kn["dim"], kn["nelem"], kn["lo"], kn["hi"], kn["p"], kn["nv"], kn["vlo"], kn["vhi"], kn["tau"],
                 bc=bc, bc_state=bcs, limiter=True, precision=FP64)
    s64.set_stream(stream.cuda_stream)
    s64.set_state(W.prim_mach5(s64.points(), cn))
    s64.step(m5["dt"], steps)
    Q64 = s64.moments().reshape(ne[0], n1, n1, n1, 5)[:, 0, 0, :, :]
    s64.close()
    m5["full_duct_moments_max_rel_diff"] = float(
        (np.abs(Qx - Q64[:, :, None, :]).max(axis=(0, 1, 2)) / moment_scales(Q64.reshape(-1, 5))).max())
    m5["full_duct_yz_homogeneity_max_abs_diff"] = float(np.abs(Qx - Qx[:, :, :1]).max())
    res["mach5"] = m5
    # Sod ensemble: one FP32-split batch, the members one after another in the FP64 form, a few against the oracle
    cb = W.config("sod_ensemble")
    members = W.sod_members(**cb)
    sol, sol64 = [], []
    for m in members:
        km = W.mesh_kwargs(m)
        for prec, lst in ((0, sol), (FP64, sol64)):
            sm = Solver(km["dim"], km["nelem"], km["lo"], km["hi"], km["p"], km["nv"], km["vlo"], km["vhi"],
                        km["tau"], bc=m["bc"], bc_state=m["bc_state"], chunks=1, precision=prec)
            sm.set_stream(stream.cuda_stream)
            sm.set_state(W.prim_sod(sm.points(), m["left"], m["right"]))
            lst.append(sm)
    dts = [sm.dt(cb["cfl"]) for sm in sol]
    b = Batch(sol)
    b.set_stream(stream.cuda_stream)
    b.autotune()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.step(dts, 1)
    b.synchronize()
    e0.record(stream)
    b.step(dts, steps - 1)
    e1.record(stream)
    b.synchronize()
    ms32 = e0.elapsed_time(e1) / max(1, steps - 1)
    for sm, dt in zip(sol64, dts):
        sm.step(dt, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for sm, dt in zip(sol64, dts):
        sm.step(dt, steps - 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / max(1, steps - 1)
    dq = 0.0
    for sm, sm64 in zip(sol, sol64):
        q32, q64 = sm.moments(), sm64.moments()
        dq = max(dq, float((np.abs(q32 - q64).max(axis=0) / moment_scales(q64)).max()))
    sod = {"members": len(members), "steps": steps, "batched_fp32_split_ms_per_step": ms32,
           "fp64_members_one_after_another_ms_per_step": ms64, "speedup_of_batched_fp32_split": ms64 / ms32,
           "moments_max_rel_diff_vs_fp64": dq}
    from oracle import oracle as orc

    do = 0.0
    for q in range(sod_oracle_members):
        m = members[q]
        km = W.mesh_kwargs(m)
        pr = orc.Problem(km["dim"], km["nelem"], km["lo"], km["hi"], km["p"], km["nv"], km["vlo"], km["vhi"],
                         km["tau"], bc=np.asarray(m["bc"]).reshape(6), bc_state=np.asarray(m["bc_state"]).reshape(6, 5))
        pr.set_state(W.prim_sod(pr.points(), m["left"], m["right"]))
        pr.step(dts[q], steps)
        qo = pr.moments()
        do = max(do, float((np.abs(sol[q].moments() - qo).max(axis=0) / moment_scales(qo)).max()))
    sod["oracle_members"] = sod_oracle_members
    sod["moments_max_rel_diff_vs_oracle"] = do
    b.close()
    for sm in sol + sol64:
        sm.close()
    res["sod_ensemble"] = sod
    # the 1-D periodic workload against the oracle (moments and f)
    c = W.config("periodic1d")
    k = W.mesh_kwargs(c)
    s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
    pr = orc.Problem(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
    prim = W.prim_field("periodic1d", pr.points())
    s.set_state(prim)
    pr.set_state(prim)
    dt = pr.dt(c["cfl"])
    s.step(dt, steps)
    pr.step(dt, steps)
    Qg, Qo = s.moments(), pr.moments()
    fg, fo = s.get_f(), pr.get_f()
    s.close()
    res["periodic1d"] = {"steps": steps, "dt": dt,
                         "moments_max_rel_diff_vs_oracle": float((np.abs(Qg - Qo).max(axis=0) / moment_scales(Qo)).max()),
                         "f_max_abs_diff_rel_vs_oracle": float(np.abs(fg - fo).max() / np.abs(fo).max())}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-baseline-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the plain all-FP64 form timed for the comparison (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="steps of the batched Sod ensemble (0: skip)")
    ap.add_argument("--mach5-steps", type=int, default=3, help="steps of the Mach-5 duct (0: skip)")
    ap.add_argument("--mach5-yz-elements", type=int, default=0,
                    help="elements in y and z of the Mach-5 duct (default: the workload's 8); narrower for profiling")
    ap.add_argument("--variant-steps", type=int, default=3,
                    help="steps of the Taylor-Green variants: limiter, variable tau, ablation (0: skip)")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--channel-steps", type=int, default=3,
                    help="steps of the full-size channel, FP32-split and all-FP64 (0: skip)")
    ap.add_argument("--curved-steps", type=int, default=3,
                    help="steps of Taylor-Green on curvilinear hexahedra (0: skip)")
    ap.add_argument("--quad-elements", type=int, default=0,
                    help="elements per direction of the planar Taylor-Green quadrilaterals (default 128)")
    ap.add_argument("--no-planar-line", action="store_true",
                    help="skip the line-element planar shear wave (profiling the quadrilaterals alone)")
    ap.add_argument("--planar-steps", type=int, default=3,
                    help="steps of the m = 2 planar shear workload (0: skip)")
    ap.add_argument("--batch-members", type=int, default=0,
                    help="members of the Sod ensemble (default: the workload's 256); smaller for profiling")
    ap.add_argument("--accuracy-steps", type=int, default=0,
                    help="steps of the per-workload accuracy comparison of the FP32-split form against the "
                         "all-FP64 GPU form and the oracle (0: skip; 100 is the stated tolerance's horizon, "
                         "about 10 minutes)")
    ap.add_argument("--elements", type=int, default=0,
                    help="elements per direction (default: the workload's 16); smaller cases for profiling")
    args = ap.parse_args()
    warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        v, sec, cores, dof, c = run_oracle(args.steps, warmup)
        sample = (f"FP64 CPU oracle, Taylor-Green field on a {c['nelem'][0]}x{c['nelem'][1]}x{c['nelem'][2]}-element "
                  f"periodic box of the benchmark's mesh spacing, p=3, full 24^3 velocity grid ({dof:.3g} DOF)")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD + " (CPU sample)", "dof": dof, "elements": list(c["nelem"]),
                           "p": c["p"], "nv": list(c["nv"])},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    __graft_entry__.build()
    from paper_2308_06196_gb300.bgk import Solver

    c = W.config(WORKLOAD)
    if args.elements:
        c = W.config(WORKLOAD, nelem=(args.elements,) * 3)
    k = W.mesh_kwargs(c)
    s = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"])
    # one non-default stream shared by the library and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream.cuda_stream)
    x = s.points()
    prim = W.prim_field(WORKLOAD, x)
    prim_pin = torch.from_numpy(prim).pin_memory()
    Q_pin = torch.empty((s.npts, 5), dtype=torch.float64).pin_memory()
    prim_dev = prim_pin.cuda()
    s.set_state(prim_dev)
    tiles_per_task = s.autotune()
    dt = s.dt(c["cfl"])
    dof = s.ndof

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (graph path and timing path)
    s.step(dt, warmup)
    s.set_timing(True)
    s.step(dt, 1)
    s.set_timing(False)
    barrier()

    # timed region: K steps through the captured CUDA graph (the library's stepping path), CUDA events
    # on the library's stream; then the same K steps launched directly, every stage and Newton launch
    # bracketed by CUDA events on its stream (the per-launch durations of the roofline). Clocks are
    # sampled during both.
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.set_state(prim_dev)
    barrier()
    with Clocks(local) as clk:
        barrier()
        g0.record(stream)
        s.step(dt, args.steps)
        g1.record(stream)
        barrier()
        s.set_state(prim_dev)
        barrier()
        s.set_timing(True)
        e0.record(stream)
        s.step(dt, args.steps)
        e1.record(stream)
        barrier()
    ms = g0.elapsed_time(g1) / args.steps
    tm = s.timing()
    s.set_timing(False)
    s.synchronize()
    event_ms = e0.elapsed_time(e1) / args.steps

    # end to end through the public API with host buffers: H2D of the primitive state, one step,
    # D2H of the moments, every step
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_state(prim_pin)
        s.step(dt, 1)
        s.moments(Q_pin)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    # the plain all-FP64 form on the same workload: time, and the FP32-split moments' distance from it
    fp64 = None
    if args.fp64_steps > 0:
        from paper_2308_06196_gb300.bgk import FP64

        s64 = Solver(k["dim"], k["nelem"], k["lo"], k["hi"], k["p"], k["nv"], k["vlo"], k["vhi"], k["tau"],
                     precision=FP64)
        s64.set_stream(stream.cuda_stream)
        s64.set_state(prim_dev)
        s64.step(dt, 1)  # warm-up (graph capture)
        s64.set_state(prim_dev)
        s.set_state(prim_dev)
        barrier()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        s64.step(dt, args.fp64_steps)
        h1.record(stream)
        barrier()
        ms64 = h0.elapsed_time(h1) / args.fp64_steps
        s.step(dt, args.fp64_steps)
        Q32, Q64 = s.moments(), s64.moments()
        # component scales: rho for mass, rho sqrt(theta) for momentum (a component of the mean
        # velocity can vanish identically), E for energy
        rho = Q64[:, 0]
        th = (2.0 / 3.0) * (Q64[:, 4] / rho - 0.5 * (Q64[:, 1:4] ** 2).sum(1) / rho**2)
        scale = np.array([rho.max()] + [(rho * np.sqrt(th)).max()] * 3 + [np.abs(Q64[:, 4]).max()])
        err = float((np.abs(Q32 - Q64).max(axis=0) / scale).max())
        fp64 = {"value": dof * 3 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
                "moments_max_rel_diff_fp32_split": err}
        s64.close()

    s.close()  # the other workloads' buffers replace the Taylor-Green ones
    variants = None
    if args.variant_steps > 0 and world == 1:
        variants = bench_variants(args.variant_steps, warmup, stream, torch, k, prim_dev, dt)
    batch = None
    if args.batch_steps > 0:
        batch = bench_batch(args.batch_steps, warmup, stream, torch, args.batch_members)
    mach5 = None
    if args.mach5_steps > 0 and world == 1:
        mach5 = bench_mach5(args.mach5_steps, warmup, stream, torch, args.mach5_yz_elements)
    ablation = None if (args.no_ablation or world > 1) else bench_ablation()
    accuracy = None
    if args.accuracy_steps > 0 and world == 1:
        accuracy = bench_accuracy(args.accuracy_steps, stream, torch)
    channel = None
    if args.channel_steps > 0 and world == 1:
        channel = bench_channel(args.channel_steps, warmup, stream, torch)
    curved = None
    if args.curved_steps > 0 and world == 1:
        curved = bench_curved(args.curved_steps, warmup, stream, torch, args.elements)
    planar = None
    if args.planar_steps > 0 and world == 1:
        planar = {} if args.no_planar_line else bench_planar(args.planar_steps, warmup, stream, torch)
        planar["quadrilaterals"] = bench_quad(args.planar_steps, warmup, stream, torch, args.quad_elements)

    ms, event_ms, e2e_ms = max_over_ranks([ms, event_ms, e2e_ms], dist, "cuda")
    value = job_value(dof, world, ms)
    e2e_value = job_value(dof, world, e2e_ms)

    stage_avg_ms = tm["stage_ms"] / max(1, tm["stage_launches"])
    achieved = tm["stage_alg_bytes"] / (stage_avg_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = stage_traffic()
    launches = tm["stage_launches"] + tm["newton_launches"]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, sec, cores, sdof, sc = run_oracle(args.cpu_baseline_steps, 1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_baseline_steps} RK3 steps of the FP64 oracle on a "
                         f"{sc['nelem'][0]}x{sc['nelem'][1]}x{sc['nelem'][2]}-element periodic Taylor-Green box "
                         f"(same spacing, p=3, 24^3 velocities, {sdof:.3g} DOF)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": f"{c['nelem'][0]}^3 hex p=3 on [0,2pi]^3", "n_x": s.npts, "nv": list(c["nv"]),
                   "dof": dof, "tau": c["tau"], "dt": dt, "precision": "f32 storage+advection, f64 Newton",
                   "l2": "inputs larger than L2 (14.5 GB per f array)", "parallelism": f"replicas x{world}",
                   "event_timed_ms_per_step": event_ms, "tiles_per_task": tiles_per_task},
        "roofline": {"bound": "hbm", "kernel": "k_stage3s", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "alg_bytes_per_launch": tm["stage_alg_bytes"], "avg_launch_ms": stage_avg_ms,
                     "stage_share": tm["stage_ms"] / (tm["stage_ms"] + tm["newton_ms"]),
                     "newton_avg_ms": tm["newton_ms"] / max(1, tm["newton_launches"])},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": s.npts * 5 * 8,
                "d2h_bytes_per_step": s.npts * 5 * 8, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "fp64_form": None if fp64 is None else dict(fp64, speedup_of_fp32_split=value / world / fp64["value"]),
        "batched": batch,
        "mach5": mach5,
        "variants": variants,
        "ablation": ablation,
        "planar": planar,
        "channel": channel,
        "curved": curved,
        "accuracy": accuracy,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
