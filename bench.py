#!/usr/bin/env python3
"""Benchmark: converged harmonic-field solves per second on the 2048x2048 scene.

One step = one pass of the planner's hot path on one synthetic 2048x2048
static scene (2000 rectangles and disks at 30 % occupancy): time-warped raster
(tw_build_grid), relaxation from the cold start u = 0.5 to the residual
r_inf <= 1e-6 with the field's error estimate held to 1e-5 (hp_relax, etol),
and the Eq. 3 path with rubber band (plan_path).

Prints one JSON line (rank 0).  `value` is device-resident throughput (inputs
already in HBM); `e2e` repeats the step through the same C ABI with host
buffers (pinned H2D of the occupancy, D2H of the field and the path) inside
the timed region, the copies on a second stream overlapping the neighbouring
steps' compute (double buffers).  Multi-GPU (torchrun): every rank solves its own scene, no
collective touches the data path; only a barrier and a max-reduce of the
elapsed time are exchanged.  `--impl reference` times the FP64 CPU oracle on
the host cores instead.
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

import scenes  # noqa: E402

METRIC = "converged-field solves/s at 2048^2, resid<=1e-6 (plus cell-updates/s vs plain FP32)"
UNIT = "solves/s"
WORKLOAD = ("static2048: 2048x2048 grid, 5 cm cells, 2000 rectangles+disks at 30% occupancy, "
            "goal (2027,2027), robot (20,20); step = raster + cold-start relaxation to r_inf<=1e-6 "
            "with the error estimate <= 1e-5 + Eq.3 path with 100 rubber-band sweeps from the robot "
            "(which returns TW_NO_PATH at once: u*(20,20) ~ 1e-12, below the field's accuracy; "
            "path_reachable times the path from a cell the field resolves)")
STORAGE_BYTES = 4           # FP32 field
MASK_BYTES = 1.0 / 8.0      # one Dirichlet bit per cell
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

# DRAM traffic of the dominant kernel from one ncu capture, valid only while
# the kernel source is unchanged (sha256 of the file that holds it).
TRAFFIC = {"ba6d59fceb4f12d5": 17464576 + 2304}   # rb_tb_kernel<7,14,12,1>, profiles/rb_tb_kernel_static2048.md


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region.

    Reads NVML in-process (libnvidia-ml through ctypes, on a helper thread)
    so no extra process competes for the driver; falls back to nvidia-smi
    when NVML cannot be loaded.  Start it before the warm-up (initialisation
    can stall the GPU context); mark_start()/mark_end() bracket the timed
    region and summary() keeps the samples taken inside it, widened by one
    sampling period on each side.
    """

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clocks-event-reason bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
               "hw_thermal_slowdown": 0x40}

    def __init__(self, gpu_index, period=0.1, mode=None):
        self.idx = gpu_index
        self.period = period
        self.mode = mode or os.environ.get("TWGRID_CLOCK_SAMPLER", "nvml")
        self.proc = None
        self.samples = []        # (time, sm_mhz, sm_max_mhz, set of reasons)
        self.t0 = self.t1 = None
        self._stop = False

    def start(self):
        if self.mode == "nvml" and self._start_nvml():
            return self
        self.mode = "nvidia-smi"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", str(int(self.period * 1000)), "-i", str(self.idx)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read_smi, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _start_nvml(self):
        import ctypes
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.idx), ctypes.byref(h)) != 0:
                return False
        except OSError:
            return False
        self.nv, self.h = nv, h
        threading.Thread(target=self._read_nvml, daemon=True).start()
        return True

    def _read_nvml(self):
        import ctypes
        cur, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop:
            ok = (self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(cur)) == 0 and
                  self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 and
                  self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(rs)) == 0)
            if ok:
                act = {n for n, b in self.REASONS.items() if rs.value & b}
                self.samples.append((time.time(), float(cur.value), float(mx.value), act))
            time.sleep(self.period)

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                act = {n for n, v in zip(names, parts[5:9]) if v.lower().startswith("active")}
                self.samples.append((time.time(), float(parts[1]), float(parts[2]), act))
            except ValueError:
                continue

    def wait_ready(self, timeout=10.0):
        t0 = time.time()
        while not self.samples and time.time() - t0 < timeout and (self.mode == "nvml" or self.proc):
            time.sleep(0.02)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        self._stop = True
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        lo = (self.t0 if self.t0 is not None else 0.0) - self.period
        hi = (self.t1 if self.t1 is not None else time.time()) + self.period
        sel = [s for s in list(self.samples) if lo <= s[0] <= hi]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": self.mode}
        reasons = set().union(*[s[3] for s in sel])
        return {"sm_mhz": statistics.median(s[1] for s in sel), "sm_max_mhz": max(s[2] for s in sel),
                "reasons": sorted(reasons), "samples": len(sel), "source": self.mode}


CLOCK_REJECT = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(c) -> str:
    """Why a timed region's clock record disqualifies it ('' if it does not):
    a hardware or thermal slowdown, or SM clocks well below their maximum with
    no reason given (a clock lock left by someone).  sw_power_cap is kept."""
    bad = sorted(set(c.get("reasons") or []) & set(CLOCK_REJECT))
    if bad:
        return ",".join(bad)
    sm, mx = c.get("sm_mhz"), c.get("sm_max_mhz")
    if sm and mx and sm < 0.8 * mx and not c.get("reasons"):
        return f"sm clock {sm:.0f} of {mx:.0f} MHz with no reason"
    return ""


def make_scene(rank: int):
    """Each rank solves its own scene (weak scaling, no data exchanged)."""
    return scenes.static2048(seed=scene_seed(rank))


def scene_seed(rank: int) -> int:
    return 1002 + 100 * rank


GOLDEN_FIELD = os.path.join(ROOT, "tests", "golden", "static2048_field.json")


def sweep_kernel_hash() -> str:
    """Hash of the source text that defines the measured sweep kernel: the tile code (hp_tile.cuh)
    and, in hp_sweeps.cu, the kernel and its tile configuration (not the host code around them),
    so that a stored ncu traffic figure is used only for the kernel it was taken on."""
    csrc = os.path.join(ROOT, "paper_1903_07441_gb300", "csrc")
    sweeps = open(os.path.join(csrc, "hp_sweeps.cu")).read()
    i = sweeps.index("template <int T, int RB, int WARPS, int MINB>")
    j = sweeps.index("};", sweeps.index("struct TBCfg", i)) + 2
    h_ = hashlib.sha256()
    h_.update(open(os.path.join(csrc, "hp_tile.cuh"), "rb").read())
    h_.update(sweeps[i:j].encode())
    return h_.hexdigest()[:16]


def field_accuracy(u, occ, sc, st):
    """The solved field against the FP64 reference u* stored for this scene
    (tests/golden/make_static2048_field.py: CG to 1e-12, exit time): the
    a-posteriori bound tau_max * r_inf and the largest error at the stored
    sample cells.  Outside the timed region."""
    import json as _json
    if not os.path.exists(GOLDEN_FIELD):
        return {"note": "no stored reference"}
    ref = _json.load(open(GOLDEN_FIELD))
    occ_h = occ.cpu().numpy()
    if (ref["nx"], ref["ny"]) != (sc.nx, sc.ny) or \
            hashlib.sha256(np.ascontiguousarray(occ_h).tobytes()).hexdigest() != ref["occupancy_sha256"]:
        return {"note": "stored reference belongs to another scene"}
    cells = np.asarray(ref["cells"], dtype=np.int64)
    ustar = np.asarray([float(v) for v in ref["u_star"]])
    got = u[cells[:, 1], cells[:, 0]].double().cpu().numpy()
    err = np.abs(got - ustar)
    out = {"reference": ref["reference"], "tau_max": ref["tau_max"], "resid_inf": st["resid_inf"],
           "error_bound": ref["tau_max"] * st["resid_inf"], "sampled_cells": int(len(cells)),
           "max_abs_error_sampled": float(err.max()), "mean_abs_error_sampled": float(err.mean()),
           "u_start": float(got[0]), "u_star_start": float(ustar[0])}
    if "descent" in ref:
        out["descent_agreement"] = descent_agreement(u, ref["descent"])
    return out


def descent_agreement(u, d):
    """Eq. 3 direction agreement where phi* > 0.99: the fraction of the stored
    sample cells (free, u* < 0.01, the reference's top two neighbours further
    apart than twice its own error bound) at which the largest of the four
    neighbours of the solved field is the reference's; overall and by u*."""
    c = np.asarray(d["cells"], dtype=np.int64)
    x, y = c[:, 0], c[:, 1]
    nb = np.stack([u[y, x + 1].cpu().numpy(), u[y, x - 1].cpu().numpy(), u[y + 1, x].cpu().numpy(),
                   u[y - 1, x].cpu().numpy()], axis=1)
    hit = np.argmax(nb, axis=1) == np.asarray(d["index"])
    us = np.asarray([float(v) for v in d["u_star"]])
    bins = {}
    for lo, hi in ((1e-3, 1e-2), (1e-4, 1e-3), (1e-5, 1e-4), (1e-6, 1e-5), (0.0, 1e-6)):
        sel = (us >= lo) & (us < hi)
        if sel.any():
            bins[f"u*[{lo:g},{hi:g})"] = {"cells": int(sel.sum()), "agree": float(hit[sel].mean())}
    return {"cells": int(len(hit)), "agree": float(hit.mean()), "by_u_star": bins,
            "free_cells_phi_above_0.99": d["free_cells_phi_above_0.99"],
            "near_ties_excluded": d["near_ties_excluded"], "reference_error_bound": d["oracle_error_bound"]}


def max_over_ranks(x: float, dist, device=None) -> float:
    """Max of a per-rank scalar (the elapsed time) over all ranks; identity without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(steps: int, world: int, elapsed_max: float) -> float:
    """Whole-job solves/s: the units all ranks processed over the slowest rank's time."""
    return steps * world / elapsed_max


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_twgrid(args, rank, world, dist):
    import torch

    import paper_1903_07441_gb300 as tw

    dev = torch.device("cuda", _env_int("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    tw.load()
    sc = make_scene(rank)
    grid = tw.make_grid(sc.nx, sc.ny, sc.cell, sc.ox, sc.oy)
    static_h = torch.from_numpy(sc.static_occ).pin_memory()
    static_d = static_h.to(dev)
    occ = torch.empty((sc.ny, sc.nx), dtype=torch.uint8, device=dev)
    u = torch.empty((sc.ny, sc.nx), dtype=torch.float32, device=dev)
    u_h = torch.empty((sc.ny, sc.nx), dtype=torch.float32).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    method = {"rbsor": tw.HP_RBSOR, "jacobi": tw.HP_JACOBI, "mixed": tw.HP_MIXED}[args.method]
    params = tw.Params(method=method, tol=args.tol, max_sweeps=args.max_sweeps, etol=args.etol,
                       tblock=args.tblock, storage={"f16": 1, "bf16": 2, "f32": 0}[args.storage])
    # the same solve with the host-driven loop and CUDA events around every batch of sweep launches
    params_timed = tw.Params(method=method, tol=args.tol, max_sweeps=args.max_sweeps, flags=tw.HP_TIMING,
                             tblock=args.tblock, storage=params.storage, etol=args.etol)
    max_len = 4 * (sc.nx + sc.ny) * 4
    stats_log = []

    def step(static_src, prm=None, field=None):
        field = u if field is None else field
        tw.tw_build_grid(grid, sc.robot, sc.tracks, sc.law, static_occ=static_src, occ=occ)
        _, st = tw.hp_relax(grid, occ, sc.goal, field=field, params=prm or params)
        pst, path = tw.plan_path(grid, field, occ, sc.start, sc.goal, rubber_iters=100, max_len=max_len)
        stats_log.append((st, pst, len(path)))
        return path

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clk = ClockSampler(dev.index).start()
    clk.wait_ready()
    # at least W warm-up steps and at least one second of them: a GPU coming out
    # of idle needs that long to reach its steady clocks
    tw0 = time.perf_counter()
    n_warm = 0
    while n_warm < args.warmup or time.perf_counter() - tw0 < args.warmup_seconds:
        flush.zero_()   # as in the timed loop: the buffer's first use costs ~0.25 s on a fresh GPU
        step(static_d)
        torch.cuda.synchronize()
        n_warm += 1
    # one step of the host-driven form timed below for the roofline: its remainder launches
    # use kernels the graph never runs, and a kernel's first launch loads its module
    step(static_d, params_timed)
    torch.cuda.synchronize()
    stats_log.clear()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_region():
        stats_log.clear()
        launches0 = tw.launch_count()
        barrier()
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
        host_ms = []
        clk.mark_start()
        ev0.record(stream)
        t0 = time.perf_counter()
        for i in range(args.steps):
            if i:
                flush.zero_()
            h0 = time.perf_counter()
            step_ev[i][0].record(stream)
            step(static_d)
            step_ev[i][1].record(stream)
            host_ms.append((time.perf_counter() - h0) * 1e3)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk.mark_end()
        # library kernels only (not the L2-flush memsets)
        return (clk.summary(), [a.elapsed_time(b) for a, b in step_ev], tw.launch_count() - launches0,
                ev0.elapsed_time(ev1) / 1e3, wall, host_ms)

    clocks, step_ms, launches, dev_s, wall, host_ms = timed_region()
    why = clocks_rejected(clocks)
    if why:   # a throttled (or clock-locked) run is measured once more
        flush.zero_()
        clocks, step_ms, launches, dev_s, wall, host_ms = timed_region()
        clocks["remeasured_after"] = why
    clk.stop()
    elapsed = max_over_ranks(max(dev_s, 1e-12), dist, dev)
    sweeps = [s["sweeps"] for s, _, _ in stats_log]
    resid = [s["resid_inf"] for s, _, _ in stats_log]
    status = [s["status"] for s, _, _ in stats_log]
    path_status = [p for _, p, _ in stats_log]
    timed_log = list(stats_log)
    # sweep-kernel launch durations: the same steps again with HP_TIMING (CUDA events
    # on the launching stream around each batch of sweep launches, host-driven loop)
    stats_log.clear()
    n_roof = max(3, min(args.steps, 10))
    for i in range(n_roof):
        if i:
            flush.zero_()
        step(static_d, params_timed)
    torch.cuda.synchronize()
    sweep_ms = sum(s["sweep_ms"] for s, _, _ in stats_log)
    sweep_launches = sum(s["sweep_launches"] for s, _, _ in stats_log)
    roof_sweeps = sum(s["sweeps"] for s, _, _ in stats_log)
    stats_log[:] = timed_log
    cells = sc.nx * sc.ny
    value = throughput(args.steps, world, elapsed)
    cups = sum(sweeps) * cells * world / elapsed

    # ---- roofline of the dominant kernel (sweep), live CUDA-event launch times
    hbm, peak_kind = peaks()
    avg_launch_s = sweep_ms / 1e3 / max(sweep_launches, 1)
    sweeps_per_launch = roof_sweeps / max(sweep_launches, 1)
    bytes_per_launch = cells * (2 * STORAGE_BYTES + MASK_BYTES) * min(1.0, sweeps_per_launch)
    achieved = bytes_per_launch / avg_launch_s / 1e9
    src_hash = sweep_kernel_hash()
    traffic = TRAFFIC.get(src_hash)
    roofline = {"bound": "hbm", "kernel": "red-black SOR sweep (hp_sweeps.cu)", "achieved": achieved,
                "peak": hbm, "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_us": avg_launch_s * 1e6, "sweeps_per_launch": sweeps_per_launch,
                "effective_cell_updates_per_s": cells * sweeps_per_launch / avg_launch_s,
                "timing": f"CUDA events on the launching stream around the sweep launches of {n_roof} "
                          "further steps of the same workload run with the host-driven loop (HP_TIMING); "
                          "the timed steps above use the graph-driven loop"}
    # the same launches against the FP32 ALU (the field pair is L2-resident at this size, so the fused
    # sweeps are bound by instruction issue rather than HBM; reported beside the contract's HBM roofline)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float((clocks or {}).get("sm_max_mhz") or 2070.0)
    alu_peak = n_sm * 128 * 2 * f_max * 1e6 / 1e12
    upd = cells * sweeps_per_launch / avg_launch_s
    roofline["alu_view"] = {"flops_per_update": 7, "achieved_tflops": 7.0 * upd / 1e12, "peak_tflops": alu_peak,
                            "frac": 7.0 * upd / 1e12 / alu_peak,
                            "peak_derivation": f"{n_sm} SMs x 128 FP32 lanes x 2 (FMA) x {f_max:.0f} MHz",
                            "note": "7 flops per useful cell-update (3 additions, then two fused multiply-adds: "
                                    "0.25 s - c and c + omega t); the Dirichlet select, the halo recomputation "
                                    "and the colour shuffles are not counted"}

    # ---- accuracy of the solved field against the stored FP64 reference of this scene
    accuracy = field_accuracy(u, occ, sc, timed_log[-1][0]) if rank == 0 else None
    if accuracy is not None:
        accuracy["err_est"] = timed_log[-1][0]["err_est"]

    # ---- the path from a start the field resolves: the robot's cell (20, 20) has u* ~ 1e-12, below the
    # accuracy of any field solved to r_inf <= 1e-6, so the step's descent returns TW_NO_PATH at once.
    # Here the descent starts from the free cell nearest the robot among those with u >= 1e-3 on the
    # step's own field (chosen outside the timed launches), and is timed with CUDA events.
    path_reachable = None
    if rank == 0:
        pick = (u >= 1e-3) & (occ == 0)
        yy, xx = torch.nonzero(pick, as_tuple=True)
        if len(yy):
            d2 = (xx - sc.start[0]) ** 2 + (yy - sc.start[1]) ** 2
            j = int(torch.argmin(d2).item())
            ps = (int(xx[j].item()), int(yy[j].item()))
            tw.plan_path(grid, u, occ, ps, sc.goal, rubber_iters=100, max_len=max_len)   # warm
            pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pms = []
            for _ in range(5):
                pa.record(stream)
                pst_, ppath = tw.plan_path(grid, u, occ, ps, sc.goal, rubber_iters=100, max_len=max_len)
                pb.record(stream)
                torch.cuda.synchronize()
                pms.append(pa.elapsed_time(pb))
            path_reachable = {"start": ps, "u_start": float(u[ps[1], ps[0]].item()), "status": int(pst_),
                              "path_len": int(len(ppath)), "ms": float(np.median(pms)),
                              "note": "plan_path (Eq. 3 descent + 100 rubber-band sweeps) from the free cell "
                                      "nearest the robot with u >= 1e-3 on the solved field; CUDA events, "
                                      "median of 5"}

    # ---- end to end through the C ABI with host buffers: every step copies its input map
    # from pinned host memory and its field back, on a copy stream with double buffers so
    # that step i's field goes back and step i+1's map comes in while step i+1 / i computes
    stats_log.clear()
    copy_s = torch.cuda.Stream(device=dev)
    u_b = [u, torch.empty_like(u)]
    st_b = [static_d, torch.empty_like(static_d)]
    uh_b = [u_h, torch.empty_like(u_h).pin_memory()]
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]
    ev_free = [torch.cuda.Event(), torch.cuda.Event()]
    barrier()
    e0 = time.perf_counter()
    ev0.record(stream)
    h2d = d2h = 0
    copy_s.wait_stream(stream)
    with torch.cuda.stream(copy_s):
        st_b[0].copy_(static_h, non_blocking=True)
        ev_in[0].record(copy_s)
    for i in range(args.steps):
        b = i & 1
        if i:
            flush.zero_()
        stream.wait_event(ev_in[b])
        if i >= 2:
            stream.wait_event(ev_free[b])   # the field buffer's previous copy-out is done
        h2d += static_h.numel() + sc.tracks.nbytes
        path = step(st_b[b], field=u_b[b])
        ev_out[b].record(stream)
        with torch.cuda.stream(copy_s):
            if i + 1 < args.steps:   # next step's input, once step i - 1 (its last reader) is done
                if i >= 1:
                    copy_s.wait_event(ev_out[1 - b])
                st_b[1 - b].copy_(static_h, non_blocking=True)
                ev_in[1 - b].record(copy_s)
            copy_s.wait_event(ev_out[b])
            uh_b[b].copy_(u_b[b], non_blocking=True)
            ev_free[b].record(copy_s)
        d2h += u_h.numel() * 4 + path.nbytes
    stream.wait_stream(copy_s)
    ev1.record(stream)
    torch.cuda.synchronize()
    assert torch.equal(uh_b[(args.steps - 1) & 1], u_b[(args.steps - 1) & 1].cpu())
    e_el = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist, dev)
    e2e = {"value": throughput(args.steps, world, e_el), "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
           "d2h_bytes_per_step": d2h // args.steps, "wall_s": time.perf_counter() - e0,
           "copies": "pinned host buffers; a copy stream overlaps step i's field copy-out and step i+1's "
                     "map copy-in with the compute (double-buffered); CUDA events around all steps"}

    # ---- plain FP32 Jacobi on the same scene (the comparison form)
    plain = None
    if not args.no_plain and rank == 0:
        pp = tw.Params(method=tw.HP_JACOBI, tol=args.tol, max_sweeps=args.plain_max_sweeps, flags=tw.HP_TIMING)
        tw.tw_build_grid(grid, sc.robot, sc.tracks, sc.law, static_occ=static_d, occ=occ)
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        _, pst = tw.hp_relax(grid, occ, sc.goal, field=u, params=pp)
        e_b.record(stream)
        torch.cuda.synchronize()
        pt = e_a.elapsed_time(e_b) / 1e3
        converged = pst["status"] == tw.TW_OK
        plain = {"method": "FP32 Jacobi (Eq. 1), 16x16 blocks, one sweep per launch", "sweeps": pst["sweeps"],
                 "converged": converged, "resid_inf": pst["resid_inf"], "seconds": pt,
                 "solves_per_s": (1.0 / pt) if converged else None,
                 "cell_updates_per_s": pst["sweeps"] * cells / pt,
                 "speedup_time_to_solution": (pt / (elapsed / args.steps)) if converged else None,
                 "note": None if converged else f"not converged within {args.plain_max_sweeps} sweeps; "
                                                 "time-to-solution is a lower bound",
                 "wall_s": time.perf_counter() - p0}

    # ---- the other forms of the relaxation on the same scene and tolerance
    forms = None
    if not args.no_forms and rank == 0:
        forms = {}
        tw.tw_build_grid(grid, sc.robot, sc.tracks, sc.law, static_occ=static_d, occ=occ)
        for name, prm in (("rbsor_fp32_graph", params),
                          ("rbsor_fp32_graph_residual_only", tw.Params(tol=args.tol, max_sweeps=args.max_sweeps)),
                          ("rbsor_fp32_host_loop", tw.Params(tol=args.tol, max_sweeps=args.max_sweeps,
                                                             flags=tw.HP_HOST_LOOP, etol=args.etol)),
                          ("rbsor_fp32_graph_polish", tw.Params(tol=args.tol, max_sweeps=args.max_sweeps,
                                                                flags=tw.HP_POLISH)),
                          ("mixed_fp16", tw.Params(method=tw.HP_MIXED, storage=tw.HP_STORE_F16, tol=args.tol,
                                                   max_sweeps=args.max_sweeps, etol=args.etol)),
                          ("mixed_bf16", tw.Params(method=tw.HP_MIXED, storage=tw.HP_STORE_BF16, tol=args.tol,
                                                   max_sweeps=args.max_sweeps, etol=args.etol)),
                          ("mixed_fp32_corrections", tw.Params(method=tw.HP_MIXED, storage=tw.HP_STORE_F32,
                                                               tol=args.tol, max_sweeps=args.max_sweeps,
                                                               etol=args.etol))):
            tw.hp_relax(grid, occ, sc.goal, field=u, params=prm)   # warm
            times, fst = [], None
            for _ in range(5):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                _, fst = tw.hp_relax(grid, occ, sc.goal, field=u, params=prm)
                b_.record(stream)
                torch.cuda.synchronize()
                times.append(a_.elapsed_time(b_))
            t_med = float(np.median(times))
            acc = field_accuracy(u, occ, sc, fst)
            forms[name] = {"ms_to_solution": t_med, "solves_per_s": 1e3 / t_med, "sweeps": fst["sweeps"],
                           "resid_inf": fst["resid_inf"], "converged": fst["status"] == tw.TW_OK,
                           "etol": prm.etol, "err_est": fst["err_est"],
                           "max_abs_error_sampled": acc.get("max_abs_error_sampled"),
                           "mean_abs_error_sampled": acc.get("mean_abs_error_sampled"),
                           "error_bound": acc.get("error_bound"),
                           "descent_agreement": (acc.get("descent_agreement") or {}).get("agree")}
            if prm.flags & tw.HP_POLISH:
                forms[name]["polishes"] = fst["polishes"]
                forms[name]["polished"] = fst["polished"]
        if plain and plain["converged"]:
            for f_ in forms.values():
                f_["speedup_vs_plain_fp32"] = plain["seconds"] * 1e3 / f_["ms_to_solution"]

    batched = run_batched(args, dev, tw) if (not args.no_batch and rank == 0) else None
    dynamic = run_dynamic(args, dev, tw) if (not args.no_dynamic and rank == 0) else None
    learned = run_learned(args, dev, tw) if (not args.no_learned and rank == 0) else None

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "method": args.method, "tol": args.tol, "etol": args.etol,
                      "parallelism": f"replicas x{world} (one scene per GPU, no collective)",
                      "l2": "256 MiB memset between timed steps (inside the timed region); the 33.5 MB "
                            "field pair itself is L2-resident within a solve"},
           "cell_updates_per_s": cups, "sweeps_per_solve": statistics.mean(sweeps) if sweeps else None,
           "resid_inf_max": max(resid) if resid else None, "relax_status": sorted(set(status)),
           "path_status": sorted(set(path_status)), "path_len": [n for _, _, n in stats_log][:1],
           "omega": stats_log[0][0]["omega"] if stats_log else None,
           "roofline": roofline, "accuracy": accuracy, "path_reachable": path_reachable, "e2e": e2e, "gpu_launches": launches, "plain_fp32": plain, "forms": forms, "batched": batched,
           "dynamic": dynamic, "learned_warm_start": learned,
           "step_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "min": min(step_ms), "max": max(step_ms), "host_p50": float(np.percentile(host_ms, 50))},
           "wall_s": wall, "clocks": clocks}
    return out


def run_batched(args, dev, tw):
    """The batched form on 256 uneven planners (side U{64..1024}, 5-35 % occupancy,
    10-300 tracks, own ring law each): per repetition, every planner's raster,
    then one hp_relax_batched call; compared with the same planners relaxed one
    by one with hp_relax."""
    import torch
    n = args.batch
    scs = [scenes.batch_fast(7000 + i) for i in range(n)]
    grids = [tw.make_grid(sc.nx, sc.ny, sc.cell) for sc in scs]
    statics = [torch.from_numpy(sc.static_occ).to(dev) for sc in scs]
    occs = [torch.empty((sc.ny, sc.nx), dtype=torch.uint8, device=dev) for sc in scs]
    fields = [torch.empty((sc.ny, sc.nx), dtype=torch.float32, device=dev) for sc in scs]
    cells = sum(sc.nx * sc.ny for sc in scs)

    def rasters():   # one by one
        for sc, g, st_, o in zip(scs, grids, statics, occs):
            tw.tw_build_grid(g, sc.robot, sc.tracks, sc.law, static_occ=st_, occ=o)

    jobs = [{"grid": g, "robot": sc.robot, "tracks": sc.tracks, "law": sc.law, "static_occ": st_, "occ": o}
            for sc, g, st_, o in zip(scs, grids, statics, occs)]

    gbatch = tw.GridBatch(jobs)

    def rasters_batched():   # all planners in one call (job table prepared once)
        gbatch.run()

    rasters()
    torch.cuda.synchronize()
    ref_occ = [o.clone() for o in occs]
    rasters_batched()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ref_occ, occs))
    del ref_occ
    torch.cuda.synchronize()
    goals = []
    for sc, o in zip(scs, occs):
        # predicted obstacles may cover the nominal goal: take the nearest free interior cell
        gx, gy = sc.goal
        if o[gy, gx].item() != 0:
            free = torch.nonzero(o[1:-1, 1:-1] == 0)
            if len(free):
                d = (free[:, 0] + 1 - gy) ** 2 + (free[:, 1] + 1 - gx) ** 2
                j = int(torch.argmin(d).item())
                gy, gx = int(free[j, 0].item()) + 1, int(free[j, 1].item()) + 1
        goals.append((gx, gy))
    # the same accuracy as the headline solve: r_inf <= tol and the error estimate <= etol
    prm = tw.Params(tol=args.tol, max_sweeps=args.max_sweeps, etol=args.etol)
    prm_res = tw.Params(tol=args.tol, max_sweeps=args.max_sweeps)
    tw.hp_relax_batched(occs, goals, fields, prm_res)   # warm: autotune + graph build
    res_times = []
    for _ in range(args.batch_reps):   # the residual test alone, for comparison
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rasters_batched()
        _, st_res, _ = tw.hp_relax_batched(occs, goals, fields, prm_res)
        b.record()
        torch.cuda.synchronize()
        res_times.append(a.elapsed_time(b) / 1e3)
    ok_res = sum(1 for st in st_res if st["status"] == tw.TW_OK)
    tw.hp_relax_batched(occs, goals, fields, prm)   # warm with the error tolerance
    stream = torch.cuda.current_stream()
    times, lats, stats, r_times = [], [], None, []
    for _ in range(args.batch_reps):
        a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        rasters_batched()
        m.record(stream)
        _, stats, lat = tw.hp_relax_batched(occs, goals, fields, prm)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
        r_times.append(a.elapsed_time(m))
        lats.extend(lat.tolist())
    t = float(np.median(times))
    # the one-by-one rasters, for comparison
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rasters()
    b.record(stream)
    torch.cuda.synchronize()
    r_seq_ms = a.elapsed_time(b)
    ok = sum(1 for st in stats if st["status"] == tw.TW_OK)
    sweeps = [st["sweeps"] for st in stats]
    updates = sum(st["sweeps"] * sc.nx * sc.ny for st, sc in zip(stats, scs))
    # the same planners one by one (single-field graph-driven solver)
    valid = [i for i, st in enumerate(stats) if st["status"] >= 0]
    for i in valid[:2]:
        tw.hp_relax(grids[i], occs[i], goals[i], field=fields[i], params=prm)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rasters()
    for i in valid:
        tw.hp_relax(grids[i], occs[i], goals[i], field=fields[i], params=prm)
    b.record(stream)
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b) / 1e3
    T = stats[0]["tblock"]
    return {"instances": n, "total_cells": cells, "converged": ok, "seconds_per_batch": t,
            "solves_per_s": ok / t, "latency_ms": {"p50": float(np.percentile(lats, 50)),
                                                 "p99": float(np.percentile(lats, 99)),
                                                 "max": float(np.max(lats))},
            "sweeps": {"min": min(sweeps), "median": float(np.median(sweeps)), "max": max(sweeps)},
            "etol": args.etol, "err_est_max": max(st["err_est"] for st in stats),
            "residual_test_only": {"solves_per_s": ok_res / float(np.median(res_times)),
                                   "seconds_per_batch": float(np.median(res_times))},
            "tblock_autotuned": T, "cell_updates_per_s": updates / t,
            "effective_gbs": updates / t * (2 * STORAGE_BYTES + MASK_BYTES) / T / 1e9,
            "sequential_seconds": t_seq, "sequential_solves_per_s": len(valid) / t_seq,
            "speedup_vs_sequential": (t_seq / max(len(valid), 1)) / (t / max(ok, 1)),
            "raster_ms": {"batched_one_call": float(np.median(r_times)), "one_by_one": r_seq_ms},
            "note": "per repetition: one tw_build_grids call (all rasters) + one hp_relax_batched call; latency = "
                    "start of the batched relaxation to each instance's convergence (device clock); the "
                    "sequential form rasters and relaxes the planners one by one"}


def run_dynamic(args, dev, tw):
    """The dynamic 512x512 configuration: 200 Kalman-tracked disks, rings 0.5 m x 1.3^j,
    100 replanning frames at 10 Hz (Kalman update + raster + warm-started relaxation
    + path + robot motion per frame), with the plain binary marking and with the
    probability-threshold marking (p_mark = 0.9)."""
    import collections

    import torch
    from paper_1903_07441_gb300 import replan
    sc = scenes.dynamic(seed=1001, side=512, n_obs=200, frames=101)
    replan.run(sc, frames=3, device=dev)   # warm
    torch.cuda.synchronize()
    out = {"workload": "dynamic512: 512x512, 5 cm, 200 moving disks (Kalman-tracked), 100 frames at 10 Hz"}
    for name, law in (("marking_binary", scenes.RingLaw()), ("marking_p0.9", scenes.RingLaw(p_mark=0.9))):
        t0 = time.perf_counter()
        res = replan.run(sc, frames=100, law=law, device=dev)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        sweeps = [f.relax.get("sweeps", 0) for f in res.frames if f.relax]
        status = collections.Counter(int(f.path_status) for f in res.frames)
        hist, edges = np.histogram(res.turning_angles(), bins=[0, 5, 10, 20, 45, 90, 180])
        out[name] = {"frames": len(res.frames), "seconds": t, "frames_per_s": len(res.frames) / t,
                     "ms_per_frame": t / max(len(res.frames), 1) * 1e3,
                     "sweeps_per_frame_median": float(np.median(sweeps)) if sweeps else None,
                     "path_ok_frames": status.get(tw.TW_OK, 0),
                     "no_path_frames": status.get(tw.TW_NO_PATH, 0),
                     "start_covered_frames": status.get(tw.TW_ESTART_BLOCKED, 0),
                     "collision_free": res.collision_free, "collision_frame": res.collision_frame,
                     "min_clearance_m": res.min_clearance, "path_length_m": res.path_length(),
                     "turning_angle_hist_deg": {f"{int(a)}-{int(b)}": int(h)
                                                for a, b, h in zip(edges[:-1], edges[1:], hist)}}
    out["note"] = ("most frames without a path end in TW_NO_PATH: the potential at the robot is 1e-11..1e-13 "
                   "through 200 obstacles and the FP64 oracle's own descent fails on these frames; relaxing longer "
                   "(500-6000 fixed sweeps per frame) does not add frames with a path; obstacles move up to 1 m/s "
                   "without avoiding the robot (0.75 m/s)")
    if args.dynamic_eval:
        out["evaluation"] = dynamic_eval(dev, tw)
    return out


def run_learned(args, dev, tw):
    """Learned warm start: the network is trained on fields the relaxation generates
    (dynamic-style 256x256 scenes: static shapes + time-warped predicted disks),
    then warm-starts the relaxation on held-out scenes at 256x256 and 1024x1024."""
    import torch

    def scene(seed, side):
        sc = scenes.dynamic(seed=seed, side=side, n_obs=12, frames=1, static_shapes=10)
        grid = tw.make_grid(side, side, sc.cell)
        occ, _ = tw.tw_build_grid(grid, sc.robot, sc.tracks, sc.law,
                                  static_occ=torch.from_numpy(sc.static_occ).to(dev))
        goal = sc.goal
        if occ[goal[1], goal[0]].item() != 0:
            goal = tw.tw_nearest_free(grid, occ, goal[0], goal[1])
        return grid, occ, goal

    side = 256
    t0 = time.perf_counter()
    data = []
    for s in range(args.learn_fields):
        grid, occ, goal = scene(20000 + s, side)
        u, _ = tw.hp_relax(grid, occ, goal, params=tw.Params(omega=1.0, tol=0.0, max_sweeps=8000))
        data.append((occ, goal, None, u))
    net = tw.WarmStartNet(dev, seed=11)
    data = [(o, g, net.target(u), None) for o, g, _, u in data]
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = []
    for it in range(args.learn_steps):
        o, g, t, _ = data[it % len(data)]
        lr = 1e-3 if it < 0.75 * args.learn_steps else 3e-4
        losses.append(net.train_step(o, g, t, lr=lr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"train_fields": len(data), "train_size": side, "train_steps": args.learn_steps,
           "data_seconds": t_gen, "train_seconds": t_train, "train_steps_per_s": args.learn_steps / t_train,
           "loss_first_100": float(np.mean(losses[:100])), "loss_last_100": float(np.mean(losses[-100:])),
           "params": net.n}
    ev = {}
    for sz, seeds in ((256, range(30000, 30008)), (1024, range(31000, 31004))):
        cold_s, cold_t = [], []
        warm = {st: ([], [], []) for st in (1, 2, 4)}   # stride -> sweeps, total ms, network ms
        for sd in seeds:
            grid, occ, goal = scene(sd, sz)
            prm = tw.Params(tol=args.tol, etol=args.etol)   # cold and warm solves to the same accuracy
            tw.hp_relax(grid, occ, goal, params=prm)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, s0 = tw.hp_relax(grid, occ, goal, params=prm)
            b.record()
            torch.cuda.synchronize()
            cold_t.append(a.elapsed_time(b))
            cold_s.append(s0["sweeps"])
            for st in (1, 2, 4):
                if sz // st < 16:
                    continue
                u0 = net.warm_start(occ, goal, st)
                a.record()
                net.warm_start(occ, goal, st, u=u0)
                m_ = torch.cuda.Event(enable_timing=True)
                m_.record()
                _, s1 = tw.hp_relax(grid, occ, goal, field=u0,
                                    params=tw.Params(tol=args.tol, etol=args.etol, flags=tw.HP_WARM_START))
                b.record()
                torch.cuda.synchronize()
                warm[st][0].append(s1["sweeps"])
                warm[st][1].append(a.elapsed_time(b))
                warm[st][2].append(a.elapsed_time(m_))
        e = {"scenes": len(cold_s), "cold_sweeps": float(np.mean(cold_s)), "cold_ms": float(np.mean(cold_t))}
        for st, (sw, tt, nt) in warm.items():
            if sw:
                e[f"stride{st}"] = {"warm_sweeps": float(np.mean(sw)), "warm_ms_incl_network": float(np.mean(tt)),
                                    "network_ms": float(np.mean(nt)),
                                    "sweep_reduction": 1.0 - float(np.mean(sw)) / float(np.mean(cold_s)),
                                    "speedup_vs_cold": float(np.mean(cold_t)) / float(np.mean(tt))}
        ev[str(sz)] = e
    out["evaluation"] = ev
    out["note"] = ("stride s: the network runs on the occupancy max-pooled by s and its prediction is "
                   "interpolated back (ws_unet_warm_start); times are CUDA events around network + relaxation")
    return out


def dynamic_eval(dev, tw, seeds=5, frames=700):
    """Success / collision-free rates and turning angles for 1-16 moving obstacles
    (the paper's Table 1 setting, on synthetic 512x512 scenes with 8 static shapes)."""
    from paper_1903_07441_gb300 import replan
    table = {}
    for n_obs in (1, 2, 4, 8, 16):
        reached = free = 0
        lengths, angles = [], []
        for k in range(seeds):
            sc = scenes.dynamic(seed=5000 + 97 * k + n_obs, side=512, n_obs=n_obs, frames=frames + 1,
                                static_shapes=8)
            res = replan.run(sc, frames=frames, device=dev)
            reached += int(res.reached)
            free += int(res.collision_free)
            lengths.append(res.path_length())
            angles.extend(res.turning_angles().tolist())
        hist, edges = np.histogram(angles, bins=[0, 5, 10, 20, 45, 90, 180])
        table[str(n_obs)] = {"runs": seeds, "reached_goal": reached, "collision_free": free,
                             "path_length_m_mean": float(np.mean(lengths)),
                             "turning_angle_hist_deg": {f"{int(a)}-{int(b)}": int(h)
                                                        for a, b, h in zip(edges[:-1], edges[1:], hist)}}
    return table


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_step(sc, max_iters=None):
    """The oracle's version of one step: brute-force raster, CG to tol, descent + band.
    Returns (seconds, cg_iterations, residual)."""
    import oracle
    t0 = time.perf_counter()
    occ, _, _ = oracle.build_grid(sc)
    u0, fixed = oracle.dirichlet_from_occ(occ, sc.goal)
    u, iters, r, _ = oracle.cg(u0, fixed, tol=1e-6, max_iters=max_iters or 1_000_000)
    oracle.plan_path(u, fixed, sc.start, sc.goal, rubber_iters=100)
    return time.perf_counter() - t0, iters, r


def cpu_baseline(sc):
    """The oracle as it stands: one full oracle step on the same scene on every host core (its
    OpenMP build, which returns the plain build's bits), and on one core."""
    import oracle
    oracle.build()
    n = os.cpu_count() or 1
    used = oracle.use_threads(n)
    try:
        t, iters, r = oracle_step(sc)
    finally:
        oracle.use_threads(1)
    t1, _, _ = oracle_step(sc)
    return {"value": 1.0 / t, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"one full oracle step on the same 2048^2 scene (brute-force raster, FP64 CG to "
                      f"r_inf<=1e-6 in {iters} iterations, descent + 100 band sweeps) on {used} threads: "
                      f"{t:.1f} s",
            "single_core": {"value": 1.0 / t1, "cores": 1, "sample": f"the same step on one core: {t1:.1f} s"}}


def run_reference(args, rank, world, dist):
    """Reference arm: the FP64 oracle on every host core (its OpenMP build; rank 0 only).  A step is
    a full oracle step when one fits the time budget, else the oracle step with a bounded number of
    CG iterations, extrapolated linearly to the iterations a full solve needs (the sample says which)."""
    import oracle
    if rank != 0:
        return None
    oracle.build()
    cores = oracle.use_threads(os.cpu_count() or 1)
    sc = make_scene(0)
    budget = max(2.0, 150.0 / max(args.steps + args.warmup, 1))
    # warm-up: one full solve to learn the CG iterations to tolerance
    t_full, n_tol, _ = oracle_step(sc)
    for _ in range(max(args.warmup - 1, 0)):
        oracle_step(sc, max_iters=5)
    m = max(5, min(n_tol, int(budget / (t_full / n_tol))))
    times = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t, iters, _ = oracle_step(sc, max_iters=m)
        times.append(t * n_tol / iters)
    total = time.perf_counter() - t0
    per_solve = statistics.mean(times)
    v = 1.0 / per_solve
    how = ("a full oracle step (raster, CG to tolerance, path)" if m >= n_tol else
           f"the oracle step with {m} of the {n_tol} CG iterations a full solve needs, extrapolated linearly")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "method": "oracle: brute-force raster + FP64 CG + descent/band"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {how}, on {cores} threads ({total:.1f} s for "
                                       f"{args.steps} steps)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_case(case):
    """One small case of a kernel other than the headline's, for an ncu capture of that kernel
    (profiles/ names the command): conv128 = a 128 -> 128 tensor-memory convolution on 512 x 512,
    conv32 = 32 -> 32 on 1024 x 1024, conv128n / conv128s = 128 -> 128 on 4096 x 64 / 64 x 64 pixels (the
    narrow form) (3 warm-up calls, then 10 timed); mixed_fp16 = one HP_MIXED FP16
    solve of a seeded 2048 x 2048 field (20 % blocked) through the host-driven loop, whose correction
    sweeps are separate launches (ncu does not profile kernel nodes of graphs with conditional nodes);
    train256 = warm-start network training steps on one 256 x 256 field (3 warm-up, 20 timed);
    wgrad128 / wgrad32 = the tensor-memory weight gradient of the conv128 / conv32 layer (3 warm-up
    calls, then 10 timed; each call adds the chunks' partial sums in a second, small kernel)."""
    import torch
    import paper_1903_07441_gb300 as tw
    dev = torch.device("cuda:0")
    if case.startswith("conv"):
        cin, cout, H, W = {"conv128": (128, 128, 512, 512), "conv32": (32, 32, 1024, 1024),
                           "conv128n": (128, 128, 4096, 64), "conv128s": (128, 128, 64, 64)}[case]
        g = torch.Generator(device=dev).manual_seed(0)
        x = (torch.randn(cin, H, W, device=dev, generator=g) * 0.5).to(torch.bfloat16)
        w = torch.randn(cout, cin, 3, 3, device=dev, generator=g) * (1.0 / (9 * cin) ** 0.5)
        b = torch.randn(cout, device=dev, generator=g) * 0.1
        for _ in range(3):
            tw.ws_conv3x3(x, w, b, relu=True, impl=tw.WS_CONV_TC)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            tw.ws_conv3x3(x, w, b, relu=True, impl=tw.WS_CONV_TC)
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / 10
        if tw.ws_conv_check():
            raise RuntimeError("a tensor-memory convolution gave up a bounded wait")
        return {"case": case, "ms_per_call": ms, "tflops": 2 * 9 * cin * cout * H * W / ms / 1e9,
                "note": "per call: the weight re-arrangement kernel and the convolution"}
    if case.startswith("wgrad"):
        cin, cout, H, W = (128, 128, 512, 512) if case == "wgrad128" else (32, 32, 1024, 1024)
        g = torch.Generator(device=dev).manual_seed(0)
        x = (torch.randn(cin, H, W, device=dev, generator=g) * 0.5).to(torch.bfloat16)
        dy = (torch.randn(cout, H, W, device=dev, generator=g) * 0.5).to(torch.bfloat16)
        for _ in range(3):
            tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_TC)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            tw.ws_conv3x3_wgrad(x, dy, impl=tw.WS_CONV_TC)
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / 10
        if tw.ws_conv_check():
            raise RuntimeError("a tensor-memory weight gradient gave up a bounded wait")
        return {"case": case, "ms_per_call": ms, "tflops": 2 * 9 * cin * cout * H * W / ms / 1e9,
                "note": "per call: two zeroed outputs, the weight-gradient kernel and the chunk sum"}
    if case == "train256":   # warm-start network training steps on one 256 x 256 field
        sc = scenes.dynamic(seed=20000, side=256, n_obs=12, frames=1, static_shapes=10)
        grid = tw.make_grid(256, 256, sc.cell)
        occ, _ = tw.tw_build_grid(grid, sc.robot, sc.tracks, sc.law, static_occ=torch.from_numpy(sc.static_occ).to(dev))
        goal = sc.goal if occ[sc.goal[1], sc.goal[0]].item() == 0 else tw.tw_nearest_free(grid, occ, *sc.goal)
        u, _ = tw.hp_relax(grid, occ, goal, params=tw.Params(omega=1.0, tol=0.0, max_sweeps=2000))
        net = tw.WarmStartNet(dev, seed=11)
        t = net.target(u)
        for _ in range(3):
            net.train_step(occ, goal, t)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(20):
            net.train_step(occ, goal, t)
        e.record()
        torch.cuda.synchronize()
        return {"case": case, "ms_per_step": a.elapsed_time(e) / 20}
    rng = np.random.default_rng(3)
    n = 2048
    occ = (rng.random((n, n)) < 0.2).astype(np.uint8)
    occ[0, :] = occ[-1, :] = occ[:, 0] = occ[:, -1] = 3
    goal = (1500, 700)
    occ[goal[1], goal[0]] = 0
    grid = tw.make_grid(n, n, 0.05)
    u, st = tw.hp_relax(grid, torch.from_numpy(occ).to(dev), goal,
                        params=tw.Params(method=tw.HP_MIXED, storage=tw.HP_STORE_F16, tol=1e-6, max_sweeps=2000,
                                         flags=tw.HP_HOST_LOOP))
    torch.cuda.synchronize()
    return {"case": case, "sweeps": st["sweeps"], "status": st["status"], "sweep_launches": st["sweep_launches"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warmup-seconds", type=float, default=3.0)
    ap.add_argument("--impl", default="twgrid", choices=["twgrid", "reference"])
    ap.add_argument("--method", default="rbsor", choices=["rbsor", "jacobi", "mixed"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--etol", type=float, default=1e-5,
                    help="error tolerance of the relaxation (hp_params.etol; 0 = the residual test alone)")
    ap.add_argument("--tblock", type=int, default=0)
    ap.add_argument("--max-sweeps", type=int, default=200000)
    ap.add_argument("--plain-max-sweeps", type=int, default=400000)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-dynamic", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learn-fields", type=int, default=1024)
    ap.add_argument("--learn-steps", type=int, default=16000)
    ap.add_argument("--dynamic-eval", action="store_true",
                    help="also run the success / collision-free evaluation over 1-16 moving obstacles")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--profile-case", choices=["conv128", "conv32", "conv128n", "conv128s", "mixed_fp16", "train256", "wgrad128",
                                                        "wgrad32"], default=None,
                    help="run one small kernel case (for an ncu capture) and print its timing, instead of the bench")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_case:
        print(json.dumps(profile_case(args.profile_case)), flush=True)
        return

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        tdist.init_process_group(backend=backend)
        dist = tdist

    if args.impl == "reference":
        out = run_reference(args, rank, world, dist)
    else:
        out = run_twgrid(args, rank, world, dist)
        if rank == 0 and world == 1 and not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(make_scene(0))
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
