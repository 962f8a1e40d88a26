"""Throughput benchmark: Fresnel target points per second at 1e-6 relative L2.

Workload (one "step" = one pass of the whole hot path): the star aperture
r = 1 + 0.3 cos 5 theta at Fresnel number 100 (lambda z = 0.0169, R = 1.3),
128 panels x 16 x 256 = 524,288 quadrature nodes regenerated every step, then
  (a) type 1: the 1000 x 1000 target grid over [-1.5, 1.5)^2 (h = 0.003), and
  (b) type 3: 1,000,000 scattered targets uniform in the disc of radius 1.5,
both in FP32 fast mode at tol 1e-6 (phases in FP64).  Metric value = 2e6
targets / step time.  Synthetic, seeded inputs (workloads.py).

The default one-GPU line also carries, each with its own step time, plan
time, roofline, error against the oracle and CPU baseline:
  fp64_path       the same star workload on the plain FP64 path (tol 1e-6);
  sweep           the 24-petal offset hyper-Gaussian starshade (Sec. 4.2) at
                  64 wavelengths in [400, 1000] nm, z = 3.7e7 m, u^oc on the
                  512 x 512 pupil grid, one batched evaluation per step
                  (wavelength sweeps per second);
  randstar_F1000  the random 20-mode aperture at Fresnel number 1000
                  (10.5M nodes) to 1e8 scattered targets in [-1.2, 1.2]^2.
Every result states its error against the oracle's direct FP64 sum on a
seeded sample of its targets, from the outputs of the last timed step; the
run exits 3 if any exceeds the tolerance.  Per-stage times come from a
separate pass with the plans' stage events on (the timed steps carry none).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload star5_F100|starshade_sweep|randstar_F1000|
                                   randstar_batch32|koch_L13] [--no-extras]
Under torchrun each rank runs an independent copy (weak scaling, no data
collective); rank 0 prints one JSON line.
"""
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

import workloads as W  # noqa: E402

METRIC = "Fresnel target pts/sec at 1e-6 rel L2 err"
UNIT = "targets/s"
TOL = 1e-6
M3 = 1_000_000
L2_FLUSH_BYTES = 512 << 20


def workload():
    cfg = W.star()
    xi, eta = W.disc_targets(M3, 1.5, 2)
    return cfg, np.ascontiguousarray(np.stack([xi, eta], 1))


SWEEP_METRIC = "starshade wavelength sweeps/sec (64 lambda, 512^2 pupil grid, 1e-6 rel L2)"
SWEEP_METRIC_N = "starshade wavelength sweeps/sec (%d lambda, 512^2 pupil grid, 1e-6 rel L2)"
SWEEP_UNIT = "sweeps/s"


def sweep_workload(n_lambda=64):
    cfg = W.starshade_sweep(n_lambda)
    g = cfg["grid"]
    gx, gy = np.meshgrid(g["h"] * np.arange(-256, 256), g["h"] * np.arange(-256, 256))
    in_pupil = int(np.count_nonzero(gx * gx + gy * gy <= cfg["pupil_radius"] ** 2))
    return cfg, in_pupil


def sweep_config(cfg, in_pupil, n_gpus):
    nl = len(cfg["problems"])
    return {"workload": "hg24_sweep%d: 24-petal HG starshade A=exp(-((r-6)/3.9)^6) on [6,14] m, "
                        "z=3.7e7 m, %d lambda in [400,1000] nm (F=13.2..5.3), u^oc on 512x512 grid "
                        "h=2.4/512 m over the pupil" % (nl, nl),
            "n_lambda": len(cfg["problems"]), "grid": "512x512", "in_pupil_targets": in_pupil,
            "tol": TOL, "precision": "fp32 spread/fft, double-float/fp64 phases",
            "nodes_recomputed_each_step": True,
            "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": "replicas x%d (independent instances, no collective)" % n_gpus}


def config_dict(cfg, n_gpus, precision="fp32"):
    g = cfg["grid"]
    return {"workload": "star5_F100: r=1+0.3cos5t, F=100 (lz=0.0169), 524288 nodes (128x16x256), "
                        "t1 1000x1000 grid h=0.003 + t3 1e6 targets in disc r<=1.5",
            "nodes": 524288, "t1_targets": g["n1"] * g["n2"], "t3_targets": M3,
            "tol": TOL,
            "precision": "fp32 spread/fft/interp, fp64 phases" if precision == "fp32" else
                         "fp64 throughout (the plain FP64 path at the same tolerance)",
            "nodes_recomputed_each_step": True,
            "streams": "t1 and t3 plans on two streams, forked and joined every step",
            "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": "replicas x%d (independent instances, no collective)" % n_gpus}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling (every 20 ms) of SM clocks and throttle reasons
    while the timed region runs.

    A reader thread timestamps each line as it arrives.  `start` returns once
    the first sample is in (so sampling is live when the timed region opens)
    and marks the region's start; `stop` marks its end, waits for one more
    sample and keeps the samples taken inside the region, plus the one just
    before it (a timed region shorter than the sampling period would
    otherwise hold none)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, index, argv=None):
        self.index = index
        self.argv = argv or ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.QUERY,
                             "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)]
        self.samples = []
        self._lines = []               # (monotonic time, fields)
        self._p = None
        self._t = None
        self._t0 = self._t1 = None

    def _read(self):
        for line in self._p.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 7:
                self._lines.append((time.monotonic(), f))

    def _wait_for(self, n, timeout):
        t_end = time.monotonic() + timeout
        while len(self._lines) < n and time.monotonic() < t_end and self._t.is_alive():
            time.sleep(0.002)

    def _launch(self, argv):
        import threading
        try:
            self._p = subprocess.Popen(argv, stdout=subprocess.PIPE,
                                       stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._p = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        self._wait_for(1, 5.0)

    def start(self):
        self._launch(self.argv)
        if self._p is not None and not self._lines and self._p.poll() is not None:
            # a sampler that rejected the short period: the common 100 ms one
            argv = [a if a != str(self.PERIOD_MS) else "100" for a in self.argv]
            if argv != self.argv:
                self.PERIOD_MS = 100
                self._launch(argv)
        self._t0 = time.monotonic()

    def stop(self):
        self._t1 = time.monotonic()
        if self._p is not None:
            n_in = sum(1 for t, _ in self._lines if t <= self._t1)
            self._wait_for(n_in + 1, 1.0)
            self._p.terminate()
            try:
                self._p.wait(timeout=10)
            except Exception:
                self._p.kill()
                self._p.wait()
            self._t.join(timeout=5)
            before = [f for t, f in self._lines if t < self._t0][-1:]
            inside = [f for t, f in self._lines if self._t0 <= t <= self._t1]
            after = [f for t, f in self._lines if t > self._t1][:1]
            # the samples bracketing the region when none fell inside it
            self.samples = before + inside if inside else before + after
        return self.summary(self._t1 - self._t0)

    def summary(self, region_s=None):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == "Active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None,
               "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
               "samples": len(self.samples), "period_ms": self.PERIOD_MS}
        if region_s is not None:
            out["timed_region_s"] = round(region_s, 4)
        return out


# ------------------------------------------------------------------ shared helpers
def _peaks():
    """(HBM GB/s, source) from the measured peaks, else the stated fallback."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except Exception:
        return 6800.0, "fallback 6800 GB/s"


def rel_error(u, ref, tol, occulter=False):
    """Relative L2 error of the aperture field u^ap against the oracle's on the
    same targets (the tolerance's meaning: an occulter output u^oc is compared
    as u^ap = 1 - u^oc, eq. bab), and the largest absolute difference (the
    paper's metric on u^oc; Babinet only flips its sign)."""
    u = np.asarray(u, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    if occulter:
        u, ref = 1.0 - u, 1.0 - ref
    d = u - ref
    rel = float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))
    return {"rel_l2": rel, "field": "u^ap = 1 - u^oc" if occulter else "u^ap",
            "max_abs": float(np.abs(d).max()) if d.size else 0.0,
            "oracle_targets": int(ref.size), "tol": tol, "within_tol": bool(rel <= tol)}


# Source files each measured kernel is built from (the DRAM traffic of an
# ncu capture holds only while these are unchanged).
KERNEL_SOURCES = {
    "spread": ["spread.cuh", "k_spread_f32.cu", "internal.cuh"],
    "interp": ["k_interp.cu", "spread.cuh", "dfloat.cuh", "internal.cuh"],
    "fft": ["k_fft.cu", "k_col_dft_tc.cu", "internal.cuh"],
    "nodes": ["k_nodes.cu", "dfloat.cuh", "internal.cuh"],
}

# Per launch, from one ncu capture of the named workload (sections
# SpeedOfLight, MemoryWorkloadAnalysis, ComputeWorkloadAnalysis, Occupancy,
# LaunchStats, SchedulerStats, WarpStateStats, InstructionStats): DRAM bytes
# read + written (dram__bytes.sum.per_second x gpu__time_duration.sum), and the
# SM-side utilisations (issue slots busy, LSU pipe, L1/TEX throughput, each a
# fraction of its own peak), with the sha256 prefix of the kernel's sources
# at the time of the capture.  A kernel whose sources changed since reports
# traffic null.
_CAP_STAR = "ncu capture of this workload (second warm-up step, every kernel)"
_CAP_SWEEP = "ncu capture of this workload (second warm-up step)"
_CAP_R1000 = "ncu capture of this workload at 3e7 targets (the spread does not depend on them)"
_SHA_SPREAD, _SHA_FFT, _SHA_INTERP = "96e6910da872462a", "6c767b5c00f7c5ff", "6d7b1b741a45e8d0"


def _cap(nbytes, issue, lsu, l1, sha, note):
    return {"bytes": nbytes, "sm_side": {"issue_slots_busy": issue, "lsu_pipe": lsu,
                                         "l1tex_throughput": l1},
            "sources_sha": sha, "note": note}


DRAM_TRAFFIC = {
    ("star5_F100", "t1.spread"): _cap(18212608, 0.487, 0.408, 0.704, _SHA_SPREAD, _CAP_STAR),
    ("star5_F100", "t3.spread"): _cap(19070208, 0.483, 0.413, 0.698, _SHA_SPREAD, _CAP_STAR),
    ("star5_F100", "t1.fft_rows"): _cap(15313152, 0.273, 0.099, 0.495, _SHA_FFT, _CAP_STAR),
    ("star5_F100", "t1.fft_cols_epilogue"): _cap(7558144, 0.230, 0.063, 0.266, _SHA_FFT,
                                                 _CAP_STAR),
    ("star5_F100", "t3.fft_rows"): _cap(6747392, 0.350, 0.126, 0.304, _SHA_FFT, _CAP_STAR),
    ("star5_F100", "t3.fft_cols"): _cap(15152384, 0.361, 0.103, 0.455, _SHA_FFT, _CAP_STAR),
    ("star5_F100", "t3.interp_epilogue"): _cap(21465344, 0.608, 0.350, 0.902, _SHA_INTERP,
                                               _CAP_STAR),
    ("hg24_sweep64", "spread"): _cap(23639579, 0.508, 0.430, 0.761, _SHA_SPREAD, _CAP_SWEEP),
    ("hg24_sweep64", "fft_rows"): _cap(16898826, 0.308, 0.104, 0.420, _SHA_FFT, _CAP_SWEEP),
    ("hg24_sweep64", "fft_cols_epilogue"): _cap(81341417, 0.393, 0.078, 0.627, _SHA_FFT,
                                                _CAP_SWEEP),
    ("randstar20_F1000", "spread"): _cap(826690109, 0.511, 0.431, 0.728, _SHA_SPREAD,
                                         _CAP_R1000),
}


def sources_sha(kind):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2010_05978_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stage_kind(stage):
    s = stage.split(".")[-1]
    if s.startswith("spread"):
        return "spread"
    if s.startswith("interp") or s == "target_sort":
        return "interp"
    if s.startswith("fft"):
        return "fft"
    if s.startswith("nodes") or s in ("scan", "scatter"):
        return "nodes"
    return None


def measured_traffic(workload_name, stage):
    """(bytes, note, SM-side utilisations) of the ncu capture of this kernel
    on this workload, or (None, why, None) when there is none or the kernel
    changed since."""
    e = DRAM_TRAFFIC.get((workload_name, stage))
    if e is None:
        return None, "no ncu capture of this kernel on this workload", None
    kind = stage_kind(stage)
    if kind is None or sources_sha(kind) != e["sources_sha"]:
        return None, "kernel sources changed since the ncu capture", None
    return e["bytes"], e["note"], e.get("sm_side")


def roofline(workload_name, ab, per_launch, note):
    """Roofline object of the stage with the largest time among those with
    algorithmic bytes: achieved = algorithmic bytes / CUDA-event time."""
    peak, src = _peaks()
    dom = max((k for k in per_launch if k in ab), key=lambda k: per_launch[k])
    achieved = ab[dom] / (per_launch[dom] * 1e-3) / 1e9
    traffic, tnote, sm_side = measured_traffic(workload_name, dom)
    out = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": traffic, "traffic_note": tnote,
           "peak_source": src, "algorithmic_bytes": ab[dom], "ms_per_launch": per_launch[dom],
           "timing": note}
    if sm_side:
        # the ceiling on the SM side: each utilisation is a fraction of its own peak (1.0)
        out["sm_side"] = dict(sm_side, ceiling=1.0, source=tnote)
    return out


def time_steps(step, stream, steps, flush=None):
    """Device time of each of `steps` calls of step(), CUDA events on the
    launching stream; an L2 flush (not timed) before each."""
    import torch
    ms = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        step()
        e.record(stream)
        e.synchronize()
        ms.append(s.elapsed_time(e))
    return ms


def stage_pass(plans, step, stream, steps, flush=None):
    """Per-stage device times (ms per step) from a separate pass with the
    plans' per-stage CUDA events on; `plans` is [(prefix, plan)].  Returns
    (stage ms per step, ms per step of this pass)."""
    for _, p in plans:
        p.set_timing(True)
    sums = {}

    def one():
        step()

    ms = []
    for _ in range(steps):
        ms += time_steps(one, stream, 1, flush)
        for pre, p in plans:
            for k, v in p.stage_times().items():
                key = pre + k
                sums[key] = sums.get(key, 0.0) + v
    for _, p in plans:
        p.set_timing(False)
    return {k: v / steps for k, v in sums.items()}, statistics.mean(ms)


def timed_plan(make):
    """A plan built by make() and its wall time with the device synchronised
    on both sides (quadrature tables, sizes, allocations, autotuning).  The
    plan is built twice and the second build timed: the first in a process
    also pays the one-time loading of the library's kernels."""
    import torch
    make().close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = make()
    torch.cuda.synchronize()
    return p, (time.perf_counter() - t0) * 1e3


# ------------------------------------------------------------------ star workload (C2)
def oracle_sample(cfg, targets, budget_s):
    """The oracle (as it stands: quadrature rebuilt + direct FP64 sum) on a
    bounded, seeded sample of the workload's targets, half on the grid and
    half scattered.  Returns its rate and its values on the sample."""
    import oracle
    from oracle import direct
    fam = cfg["families"]
    g = cfg["grid"]
    gx, gy = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    rng = W.rng(2, 11)
    x, y, w = oracle.nodes(fam)                       # calibration only
    t0 = time.perf_counter()
    direct.direct_sum(x, y, w, gx[:64], gy[:64], cfg["lam"] * cfg["z"])
    per_target = max((time.perf_counter() - t0) / 64, 1e-7)
    m = int(max(16, min(200000, budget_s / per_target)))
    m -= m % 2
    ig = np.sort(rng.choice(len(gx), m // 2, replace=False))
    it = np.sort(rng.choice(len(targets), m // 2, replace=False))
    xi = np.concatenate([gx[ig], targets[it, 0]])
    eta = np.concatenate([gy[ig], targets[it, 1]])
    t0 = time.perf_counter()
    u = oracle.field(fam, cfg["lam"], cfg["z"], xi, eta)
    dt = time.perf_counter() - t0
    rate = {"value": m / dt, "unit": UNIT, "cores": direct.max_threads(), "kind": "oracle",
            "sample": "%d targets (%d grid + %d scattered) of the same workload, quadrature "
                      "rebuilt + direct O(NM) FP64 sum (eq. faq), %.1f s" % (m, m // 2, m // 2, dt)}
    return {"rate": rate, "ig": ig, "it": it, "ref1": u[: m // 2], "ref3": u[m // 2:]}


def star_error(out1, out3, sample, tol, bar=None):
    """Errors of the star step's outputs on the oracle sample; within_tol
    compares them with bar (the mode's stated bound: tol itself in the fast
    mode, 1e-10 for FP64 at tol 1e-12)."""
    import torch
    bar = tol if bar is None else bar
    u1 = out1.reshape(-1)[torch.as_tensor(sample["ig"], device=out1.device)]
    u3 = out3[torch.as_tensor(sample["it"], device=out3.device)]
    u1, u3 = u1.cpu().numpy(), u3.cpu().numpy()
    e1 = rel_error(u1, sample["ref1"], bar)
    e3 = rel_error(u3, sample["ref3"], bar)
    return {"t1_rel_l2": e1["rel_l2"], "t3_rel_l2": e3["rel_l2"],
            "max_abs_uoc": max(e1["max_abs"], e3["max_abs"]),
            "oracle_targets": e1["oracle_targets"] + e3["oracle_targets"], "tol": tol,
            "bar": bar, "within_tol": e1["within_tol"] and e3["within_tol"],
            "against": "the oracle's direct FP64 sum (eq. faq) on its own quadrature, on the "
                       "cpu_baseline sample's targets; outputs of the last timed step"}


def star_arm(args, dev, local_rank, world, precision, steps, warmup, sample=None, e2e=True,
             tol=TOL, bar=None):
    """Times the star workload (type 1 on the 1000^2 grid + type 3 on 1e6
    scattered targets, nodes regenerated every step) in one precision at
    tolerance tol."""
    import torch
    from paper_2010_05978_gb300 import Plan
    cfg, targets_np = workload()
    fam, g = cfg["families"], cfg["grid"]
    stream = torch.cuda.current_stream()
    # the type-1 and type-3 evaluations are independent: each plan has its
    # own stream and a step forks the second off the first and joins it back
    stream3 = torch.cuda.Stream()
    cdt = star_cdtype(torch, precision)
    targets = torch.tensor(targets_np, dtype=torch.float64, device=dev)
    det = bool(getattr(args, "deterministic", False))
    p1, ms1 = timed_plan(lambda: Plan(fam, cfg["lam"], cfg["z"], tol, precision=precision, grid=g,
                                      recompute_nodes=True, sync_status=False,
                                      deterministic=det))
    p3, ms3 = timed_plan(lambda: Plan(fam, cfg["lam"], cfg["z"], tol, precision=precision,
                                      box=(-1.5, 1.5, -1.5, 1.5), recompute_nodes=True,
                                      sync_status=False, stream=stream3, deterministic=det))
    info1, info3 = p1.info(), p3.info()
    out1 = torch.empty((g["n2"], g["n1"]), dtype=cdt, device=dev)
    out3 = torch.empty((M3,), dtype=cdt, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        stream3.wait_stream(stream)
        p1.eval(None, out1)
        p3.eval(targets, out3)
        stream.wait_stream(stream3)

    def step_serial():
        p1.eval(None, out1)
        stream3.wait_stream(stream)
        p3.eval(targets, out3)
        stream.wait_stream(stream3)

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    p1.check()
    p3.check()
    clocks = ClockSampler(local_rank) if local_rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    step_ms = time_steps(step, stream, steps, flush)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    p1.check()
    p3.check()
    ms_per_step, value = aggregate_ranks(sum(step_ms), steps, 2e6, world, dev)
    err = star_error(out1, out3, sample, tol, bar) if sample is not None else None
    stages, stage_step_ms = stage_pass([("t1.", p1), ("t3.", p3)], step_serial, stream,
                                       max(3, min(steps, 10)), flush)
    res = {"ms_per_step": ms_per_step, "value": value, "plan_ms": ms1 + ms3,
           "plan_plus_eval_ms": ms1 + ms3 + ms_per_step, "error": err,
           "stages_ms_per_step": {k: round(v, 5) for k, v in sorted(stages.items())},
           "stage_pass_ms_per_step": stage_step_ms,
           "launches_per_step": info1["launches_per_eval"] + info3["launches_per_eval"],
           "step_ms_median": statistics.median(step_ms), "step_ms_best": min(step_ms),
           "clocks": clk, "info": (info1, info3)}
    ab = algorithmic_bytes(info1, info3, info1["n_nodes"], precision)
    res["roofline"] = roofline("star5_F100" if precision == "fp32" else "star5_F100_fp64", ab,
                               stages, "stage pass: per-stage CUDA events on each plan's stream, "
                               "type 1 then type 3 serialised (no overlap), %d steps; the headline "
                               "step is timed without stage events" % max(3, min(steps, 10)))
    if e2e:
        # end to end through the C ABI with host buffers: pinned host arrays
        # in and out, host<->device copies inside the timed region; each step
        # ends with one device synchronisation.
        h_t3 = torch.from_numpy(targets_np).pin_memory().numpy()
        h_out1 = torch.empty((g["n2"], g["n1"]), dtype=cdt, pin_memory=True).numpy()
        h_out3 = torch.empty((M3,), dtype=cdt, pin_memory=True).numpy()
        for _ in range(2):
            p1.eval_host(None, h_out1)
            p3.eval_host(h_t3, h_out3)
            torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(max(3, min(steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p1.eval_host(None, h_out1)
            p3.eval_host(h_t3, h_out3)
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        p1.check()
        p3.check()
        res["e2e"] = {"value": 2e6 * world / (statistics.median(e2e_ms) * 1e-3), "unit": UNIT,
                      "h2d_bytes_per_step": int(h_t3.nbytes),
                      "d2h_bytes_per_step": int(h_out1.nbytes + h_out3.nbytes)}
    p1.close()
    p3.close()
    return res


def live_rows(info, full):
    """Grid rows a type-1 plan spreads and transforms: its live tile rows
    (those holding nodes) times the tile height, else every row."""
    lr = info.get("live_tile_rows", 0)
    return min(full, lr * info.get("tile_y", 32)) if lr > 0 else full


def algorithmic_bytes(info1, info3, n_nodes, precision="fp32"):
    """Minimum bytes each stage must move, per launch.  FP32 fast mode: a
    24 B node record (2 x int32 cell, 2 x f32 fraction, c64 strength) and c64
    grids; FP64 mode: a 40 B record (f64 fractions, c128 strength) and c128.
    Type 1 counts only the live rows of its spreading grid (the passes skip
    rows that hold no nodes)."""
    rec = 24 if precision == "fp32" else 40
    c64 = 8 if precision == "fp32" else 16
    nf1, nf2 = info1["nf1"], info1["nf2"]
    r1 = live_rows(info1, nf2)
    g3 = info3["nf1"] * info3["nf2"]
    F3 = info3["nfft1"] * info3["nfft2"]
    return {
        # t1
        "t1.spread": n_nodes * rec + nf1 * r1 * c64,
        "t1.fft_rows": nf1 * r1 * c64 + 1000 * r1 * c64,
        "t1.fft_cols_epilogue": 1000 * r1 * c64 + 1000 * 1000 * c64,
        # t3
        "t3.spread": n_nodes * rec + g3 * c64,
        "t3.fft_rows": g3 * c64 + info3["nf2"] * info3["nfft1"] * c64,
        "t3.fft_cols": info3["nf2"] * info3["nfft1"] * c64 + F3 * c64,
        "t3.interp_epilogue": M3 * (16 + c64),
    }


def star_cdtype(torch, precision):
    return torch.complex64 if precision == "fp32" else torch.complex128


def run_reference(args, rank, world):
    cfg, targets = workload()
    from oracle import build as obuild
    obuild.build()
    if rank != 0:
        return
    budget = 6.0
    for _ in range(args.warmup):
        oracle_sample(cfg, targets, 0.5)
    vals = []
    for _ in range(args.steps):
        r = oracle_sample(cfg, targets, budget)["rate"]
        vals.append(r["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 2e6 / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(cfg, args.gpus, args.precision),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def aggregate_ranks(total_ms, steps, units_per_step, world, device="cpu"):
    """Weak scaling over independent replicas: every rank processed
    units_per_step per step; the job's time is the slowest rank's (max over
    ranks, the only collective).  Returns (ms per step, job units per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / steps
    return ms_per_step, units_per_step * world / (ms_per_step * 1e-3)


def _setup(rank, world, local_rank):
    import torch
    from paper_2010_05978_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        build.build()
    torch.cuda.set_device(local_rank)
    return torch.device("cuda", local_rank)


def _compact(res, keys=("ms_per_step", "value", "plan_ms", "plan_plus_eval_ms", "error",
                        "roofline", "stages_ms_per_step", "clocks")):
    return {k: res[k] for k in keys if k in res}


def run_ours(args, rank, world, local_rank):
    """The headline line: the star workload in FP32 fast mode.  At one GPU the
    same line also carries the plain FP64 path on the same workload and
    tolerance, the 64-wavelength starshade sweep and the F = 1000 random
    aperture with 1e8 targets, each with its own timing, roofline, error
    against the oracle and CPU baseline."""
    dev = _setup(rank, world, local_rank)
    prec = args.precision
    cfg, targets_np = workload()
    sample = None
    if rank == 0:
        from oracle import build as obuild
        obuild.build()
        # the oracle on a bounded sample: the CPU baseline, and the reference
        # values the GPU outputs of the timed steps are checked against
        sample = oracle_sample(cfg, targets_np, 8.0)
    main = star_arm(args, dev, local_rank, world, prec, args.steps, args.warmup, sample)
    extras = {}
    if world == 1 and args.extras and prec == "fp32" and not args.deterministic:
        f64 = star_arm(args, dev, local_rank, world, "fp64", min(args.steps, 20), 3, sample,
                       e2e=False)
        extras["fp64_path"] = dict(_compact(f64), precision="fp64 throughout, tol 1e-6",
                                   fp32_speedup=main["value"] / f64["value"])
        # the paper's own precision: FP64 at tol 1e-12 (bar 1e-10)
        f64p = star_arm(args, dev, local_rank, world, "fp64", min(args.steps, 10), 3, sample,
                        e2e=False, tol=1e-12, bar=1e-10)
        extras["fp64_tol_1e-12"] = dict(_compact(f64p),
                                        precision="fp64 throughout, tol 1e-12 (bar 1e-10)",
                                        kernel={"w": f64p["info"][0]["w"],
                                                "sigma": f64p["info"][0]["sigma"]})
        extras["sweep"] = sweep_arm(args, dev, local_rank, 1, 64, args.steps, args.warmup,
                                    budget_s=5.0)
        extras["randstar_F1000"] = randstar_arm(args, dev, local_rank, 1, False,
                                                min(args.steps, 10), 3, budget_s=5.0)
    if rank != 0:
        return
    info1, info3 = main["info"]
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": main["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "step_ms_median": main["step_ms_median"], "step_ms_best": main["step_ms_best"],
        "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": dict(config_dict(cfg, world, prec),
                       **({"deterministic": "exact fixed-point spreading (bitwise-repeatable)"}
                          if args.deterministic else {})),
        "roofline": main["roofline"],
        "error": main["error"],
        "plan_ms": main["plan_ms"], "plan_plus_eval_ms": main["plan_plus_eval_ms"],
        "stages_ms_per_step": main["stages_ms_per_step"],
        "stage_pass_ms_per_step": main["stage_pass_ms_per_step"],
        "cpu_baseline": sample["rate"],
        "e2e": main["e2e"],
        "gpu_launches": main["launches_per_step"] * args.steps,
        "clocks": main["clocks"],
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    bad = [k for k, v in [("star", line["error"])] + [(k, e.get("error")) for k, e in extras.items()]
           if v is not None and not v["within_tol"]]
    if bad:
        sys.stderr.write("error above tolerance in: %s\n" % ", ".join(bad))
        sys.exit(3)


# ------------------------------------------------------------------ starshade sweep (C3)
def sweep_oracle_sample(cfg, budget_s):
    """Oracle sweeps/s: direct sums of three wavelengths on sampled grid
    targets, scaled to the full sweep (64 wavelengths x 512^2 targets); its
    values on the sample are returned for the error of the GPU sweep."""
    import oracle
    from oracle import direct
    g = cfg["grid"]
    gx, gy = oracle.grid_targets(g["n1"], g["n2"], g["h"])
    nb = len(cfg["problems"])
    which = (0, nb // 2, nb - 1)
    rng = W.rng(3, 21)
    q = cfg["problems"][0]
    t0 = time.perf_counter()
    oracle.field(q["families"], q["lam"], q["z"], gx[:32], gy[:32])
    per = max((time.perf_counter() - t0) / 32, 1e-7)
    m = int(max(16, min(100000, budget_s / per / len(which))))
    t_total, n_total, refs = 0.0, 0, []
    for b in which:
        q = cfg["problems"][b]
        idx = np.sort(rng.choice(len(gx), m, replace=False))
        t0 = time.perf_counter()
        u = oracle.field(q["families"], q["lam"], q["z"], gx[idx], gy[idx], output="occulter")
        t_total += time.perf_counter() - t0
        n_total += m
        refs.append((b, idx, u))
    per_target = t_total / n_total
    sweep_s = per_target * len(gx) * nb   # the whole sweep
    rate = {"value": 1.0 / sweep_s, "unit": SWEEP_UNIT, "cores": direct.max_threads(),
            "kind": "oracle",
            "sample": "%d grid targets at each of 3 wavelengths (400, ~700, 1000 nm), quadrature "
                      "rebuilt + direct O(NM) FP64 sum (eq. faq), %.1f s; scaled to %d x 512^2"
                      % (m, t_total, nb)}
    return rate, refs


def sweep_arm(args, dev, local_rank, world, n_lambda, steps, warmup, budget_s=10.0):
    import torch
    from paper_2010_05978_gb300 import BatchPlan
    cfg, in_pupil = sweep_workload(n_lambda)
    g = cfg["grid"]
    B = len(cfg["problems"])
    stream = torch.cuda.current_stream()
    p, plan_ms = timed_plan(lambda: BatchPlan(cfg["problems"], TOL, precision="fp32", grid=g,
                                              output="occulter", recompute_nodes=True,
                                              sync_status=False))
    info = p.info()
    out = torch.empty((B, g["n2"], g["n1"]), dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(warmup, 3)):
        p.eval(out=out)
    torch.cuda.synchronize()
    p.check()
    clocks = ClockSampler(local_rank) if local_rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    step_ms = time_steps(lambda: p.eval(out=out), stream, steps, flush)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    p.check()
    ms_per_step, value = aggregate_ranks(sum(step_ms), steps, 1.0, world, dev)
    cpu, refs, err = None, None, None
    if local_rank == 0:
        cpu, refs = sweep_oracle_sample(cfg, budget_s)
        us = np.concatenate([out[b].reshape(-1)[torch.as_tensor(idx, device=dev)].cpu().numpy()
                             for b, idx, _ in refs])
        ref = np.concatenate([u for _, _, u in refs])
        e = rel_error(us, ref, TOL, occulter=True)
        err = dict(e, against="the oracle's direct FP64 sum (eq. faq) on its own quadrature, "
                              "u^oc at sampled grid targets of 3 wavelengths (400, ~700, 1000 nm); "
                              "outputs of the last timed step")
    stages, stage_ms = stage_pass([("", p)], lambda: p.eval(out=out), stream,
                                  max(3, min(steps, 10)), flush)

    # end to end: the same call plus the read-back of every field to pinned host memory
    h_out = torch.empty((B, g["n2"], g["n1"]), dtype=torch.complex64, pin_memory=True)
    e2e_ms = []
    for i in range(max(3, min(steps, 10)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.eval(out=out)
        h_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        if i:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    c64, rec = 8, 24
    nf1, nf2, n1, n2 = info["nf1"], info["nf2"], g["n1"], g["n2"]
    rows = live_rows(info, B * nf2)   # grid rows the pruned passes spread and transform
    ab = {"spread": info["n_nodes"] * rec + rows * nf1 * c64,
          "fft_rows": rows * (nf1 + n1) * c64,
          "fft_cols_epilogue": (rows * n1 + B * n1 * n2) * c64}
    res = {"metric": SWEEP_METRIC_N % B, "unit": SWEEP_UNIT, "ms_per_step": ms_per_step,
           "value": value, "plan_ms": plan_ms, "plan_plus_eval_ms": plan_ms + ms_per_step,
           "targets_per_s": value * B * in_pupil, "error": err,
           "config": sweep_config(cfg, in_pupil, world),
           "roofline": roofline("hg24_sweep%d" % B, ab, stages,
                                "stage pass: per-stage CUDA events, %d steps; the sweep step is "
                                "timed without stage events" % max(3, min(steps, 10))),
           "stages_ms_per_step": {k: round(v, 5) for k, v in sorted(stages.items())},
           "stage_pass_ms_per_step": stage_ms,
           "cpu_baseline": cpu,
           "e2e": {"value": world / (statistics.median(e2e_ms) * 1e-3), "unit": SWEEP_UNIT,
                   "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(h_out.numel() * 8)},
           "gpu_launches": info["launches_per_eval"] * steps, "clocks": clk,
           "steps": steps}
    p.close()
    # the same sweep with the quadrature, chirp and binning done once at plan
    # time (the paper gives sweep times with and without building the
    # quadrature): spread, FFT and epilogue per step
    q = BatchPlan(cfg["problems"], TOL, precision="fp32", grid=g, output="occulter",
                  recompute_nodes=False, sync_status=False)
    for _ in range(3):
        q.eval(out=out)
    torch.cuda.synchronize()
    c_ms = time_steps(lambda: q.eval(out=out), stream, steps, flush)
    q.check()
    c_per, c_value = aggregate_ranks(sum(c_ms), steps, 1.0, world, dev)
    res["nodes_cached"] = {"ms_per_step": c_per, "value": c_value, "unit": SWEEP_UNIT,
                           "launches_per_step": q.info()["launches_per_eval"]}
    q.close()
    # the same sweep at the paper's precision: FP64 throughout at tol 1e-12
    # (bar 1e-10), nodes rebuilt every step
    d = BatchPlan(cfg["problems"], 1e-12, precision="fp64", grid=g, output="occulter",
                  recompute_nodes=True, sync_status=False)
    out64 = torch.empty((B, g["n2"], g["n1"]), dtype=torch.complex128, device=dev)
    for _ in range(3):
        d.eval(out=out64)
    torch.cuda.synchronize()
    d_ms = time_steps(lambda: d.eval(out=out64), stream, max(3, min(steps, 10)), flush)
    d.check()
    d_per, d_value = aggregate_ranks(sum(d_ms), len(d_ms), 1.0, world, dev)
    e64 = None
    if refs is not None:
        us64 = np.concatenate([out64[b].reshape(-1)[torch.as_tensor(idx, device=dev)].cpu().numpy()
                               for b, idx, _ in refs])
        e64 = rel_error(us64, ref, 1e-10, occulter=True)
    res["fp64_tol_1e-12"] = {"ms_per_step": d_per, "value": d_value, "unit": SWEEP_UNIT,
                             "error": e64, "kernel": {"w": d.info()["w"],
                                                      "sigma": d.info()["sigma"]}}
    d.close()
    del out64
    return res


def run_sweep(args, rank, world, local_rank):
    dev = _setup(rank, world, local_rank)
    if rank == 0:
        from oracle import build as obuild
        obuild.build()
    r = sweep_arm(args, dev, local_rank, world, args.lambdas, args.steps, args.warmup)
    if rank != 0:
        return
    line = {"metric": r["metric"], "value": r["value"], "unit": SWEEP_UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": r["config"]}
    line.update({k: v for k, v in r.items() if k not in line and k not in ("metric", "steps")})
    print(json.dumps(line), flush=True)


def run_sweep_reference(args, rank, world):
    cfg, in_pupil = sweep_workload(args.lambdas)
    from oracle import build as obuild
    obuild.build()
    if rank != 0:
        return
    for _ in range(args.warmup):
        sweep_oracle_sample(cfg, 0.3)
    vals = [sweep_oracle_sample(cfg, 6.0)[0]["value"] for _ in range(args.steps)]
    r = sweep_oracle_sample(cfg, 1.0)[0]
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": SWEEP_METRIC_N % args.lambdas, "value": v,
            "unit": SWEEP_UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": sweep_config(cfg, in_pupil, args.gpus),
            "cpu_baseline": {"value": v, "unit": SWEEP_UNIT, "cores": r["cores"],
                             "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": v, "unit": SWEEP_UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ F = 1000 random aperture (C5)
R1000_METRIC = "Fresnel target pts/sec at 1e-6 rel L2 err (F=1000, 1e7 nodes, 1e8 scattered targets)"
BATCH_METRIC = "Fresnel target pts/sec at 1e-6 rel L2 err (32-instance batch, 1e5-2e6 nodes, 5.5e7 targets)"


def _host_targets(counts, config_id, streams):
    xs, ys = [], []
    for m, st in zip(counts, streams):
        x, y = W.square_targets(m, 1.2, config_id, st)
        xs.append(x)
        ys.append(y)
    return np.ascontiguousarray(np.stack([np.concatenate(xs), np.concatenate(ys)], 1))


def _oracle_rate_t3(problems, targets_per, budget_s):
    """Oracle targets/s on a bounded sample: a few targets of each problem,
    quadrature rebuilt + direct FP64 sum; returns the values too (None for
    problems the budget left out)."""
    import oracle
    from oracle import direct
    t_total, n_total, refs = 0.0, 0, []
    for q, (x, y) in zip(problems, targets_per):
        if t_total > budget_s:
            refs.append(None)
            continue
        t0 = time.perf_counter()
        refs.append(oracle.field(q["families"], q["lam"], q["z"], x, y))
        t_total += time.perf_counter() - t0
        n_total += len(x)
    return n_total / t_total, direct.max_threads(), n_total, t_total, refs


def randstar_arm(args, dev, local_rank, world, batch, steps, warmup, budget_s=10.0):
    import torch
    from paper_2010_05978_gb300 import BatchPlan, Plan
    box = (-1.2, 1.2, -1.2, 1.2)
    if batch:
        problems, counts = W.random_star_batch()
        h_t = _host_targets(counts, 5, [100 + i for i in range(len(counts))])
        p, plan_ms = timed_plan(lambda: BatchPlan(problems, TOL, precision="fp32", box=box,
                                                  recompute_nodes=True, sync_status=False))
        step = lambda t, o: p.eval(t, counts, o)
        metric, name = BATCH_METRIC, "randstar_batch32"
    else:
        cfg = W.random_star()
        problems = [{"families": cfg["families"], "lam": cfg["lam"], "z": cfg["z"]}]
        counts = [int(getattr(args, "targets", 0) or 100_000_000)]
        h_t = _host_targets(counts, 5, [1])
        p, plan_ms = timed_plan(lambda: Plan(cfg["families"], cfg["lam"], cfg["z"], TOL,
                                             precision="fp32", box=box, recompute_nodes=True,
                                             sync_status=False))
        step = lambda t, o: p.eval(t, o)
        metric, name = R1000_METRIC, "randstar20_F1000"
    total = sum(counts)
    info = p.info()
    t = torch.from_numpy(h_t).to(dev)
    out = torch.empty(total, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(warmup, 3)):
        step(t, out)
    torch.cuda.synchronize()
    p.check()
    clocks = ClockSampler(local_rank) if local_rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    # inputs (1.6 GB / 0.9 GB of targets) are larger than L2: no flush
    step_ms = time_steps(lambda: step(t, out), stream, steps)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    p.check()
    ms_per_step, value = aggregate_ranks(sum(step_ms), steps, float(total), world, dev)
    # the oracle on a bounded sample of the same targets: CPU baseline and error
    cpu, err = None, None
    if local_rank == 0:
        sample, offs = [], []
        off = 0
        for i, m in enumerate(counts):
            idx = np.sort(W.rng(5, 900 + i).choice(m, 8 if batch else 200, replace=False))
            sample.append((h_t[off + idx, 0], h_t[off + idx, 1]))
            offs.append(off + idx)
            off += m
        rate, cores, n_s, t_s, refs = _oracle_rate_t3(problems, sample, budget_s)
        keep = [i for i, r in enumerate(refs) if r is not None]
        gidx = np.concatenate([offs[i] for i in keep])
        ref = np.concatenate([refs[i] for i in keep])
        u = out[torch.as_tensor(gidx, device=dev)].cpu().numpy()
        err = dict(rel_error(u, ref, TOL),
                   against="the oracle's direct FP64 sum (eq. faq) on its own quadrature at "
                           "sampled targets; outputs of the last timed step")
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d targets of the same instances, quadrature rebuilt + direct O(NM) "
                         "FP64 sum (eq. faq), %.1f s" % (n_s, t_s)}
    stages, stage_ms = {}, None
    if not batch:   # stage times are not kept inside the batch's captured graph
        stages, stage_ms = stage_pass([("", p)], lambda: step(t, out), stream, 3)
    unbatched = None
    if batch:
        # the same instances as separate plans evaluated one after another on
        # one stream: what the batch (one captured graph over four streams)
        # replaces
        singles = [Plan(q["families"], q["lam"], q["z"], TOL, precision="fp32", box=box,
                        recompute_nodes=True, sync_status=False) for q in problems]
        offs = np.concatenate([[0], np.cumsum(counts)])

        def seq():
            for i, q in enumerate(singles):
                singles[i].eval(t[offs[i]:offs[i + 1]], out[offs[i]:offs[i + 1]])
        for _ in range(2):
            seq()
        torch.cuda.synchronize()
        seq_ms = statistics.median(time_steps(seq, stream, max(3, min(steps, 5))))
        for q in singles:
            q.close()
        unbatched = {"ms_per_step": seq_ms, "value": total / (seq_ms * 1e-3),
                     "how": "the same %d instances as separate plans, evaluated one after "
                            "another on one stream" % len(problems)}
        # the same batch with the upsampling factor 1.5 instead of 2 (the
        # option fresnel_opts.sigma): 0.56 x the FFT cells for a wider
        # kernel, and a larger FP32 error (the deconvolution amplifies the
        # rounding more), so not the default
        q15 = BatchPlan(problems, TOL, precision="fp32", box=box, recompute_nodes=True,
                        sync_status=False, sigma=1.5)
        out15 = torch.empty_like(out)
        for _ in range(2):
            q15.eval(t, counts, out15)
        torch.cuda.synchronize()
        s15 = statistics.median(time_steps(lambda: q15.eval(t, counts, out15), stream,
                                           max(3, min(steps, 5))))
        q15.check()
        e15 = None
        if local_rank == 0:
            e15 = rel_error(out15[torch.as_tensor(gidx, device=dev)].cpu().numpy(), ref, TOL)
        sigma15 = {"ms_per_step": s15, "value": total / (s15 * 1e-3), "error": e15,
                   "kernel": {"w": q15.info()["w"], "sigma": q15.info()["sigma"]}}
        q15.close()
        del out15
    # end to end: host targets in, host fields out, inside the timed region
    h_out = torch.empty(total, dtype=torch.complex64, pin_memory=True)
    h_in = torch.from_numpy(h_t).pin_memory()
    e2e_ms = []
    for i in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t.copy_(h_in, non_blocking=True)
        step(t, out)
        h_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        if i:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = total * world / (statistics.median(e2e_ms) * 1e-3)
    peak, src = _peaks()
    c64 = 8
    if batch:
        ab = total * (16 + c64) + info["n_nodes"] * 24
        roof = {"bound": "hbm", "kernel": "whole batch step (one graph)", "achieved":
                ab / (ms_per_step * 1e-3) / 1e9, "algorithmic_bytes": ab,
                "ms_per_launch": ms_per_step, "peak": peak, "unit": "GB/s",
                "frac": ab / (ms_per_step * 1e-3) / 1e9 / peak, "traffic": None,
                "traffic_note": "whole step, not one kernel", "peak_source": src,
                "timing": "the timed steps"}
    else:
        g = info["nf1"] * info["nf2"]
        F = info["nfft1"] * info["nfft2"]
        ab = {"spread": info["n_nodes"] * 24 + g * c64,
              "fft_rows": (g + info["nf2"] * info["nfft1"]) * c64,
              "fft_cols": (info["nf2"] * info["nfft1"] + F) * c64,
              "interp_epilogue": total * (16 + c64)}
        if "target_sort" in stages:   # binned interpolation: targets read, permutation written
            ab["target_sort"] = total * (16 + 4)
        roof = roofline(name, ab, stages, "stage pass: per-stage CUDA events, 3 steps; the "
                        "headline step is timed without stage events")
    res = {"metric": metric, "unit": UNIT, "ms_per_step": ms_per_step, "value": value,
           "plan_ms": plan_ms, "plan_plus_eval_ms": plan_ms + ms_per_step, "error": err,
           "config": {"workload": name, "targets": total, "nodes": info["n_nodes"],
                      "instances": len(problems), "tol": TOL,
                      "precision": "fp32 spread/fft/interp, double-float phases",
                      "nodes_recomputed_each_step": True,
                      "l2": "inputs larger than L2 (targets %.1f GB)" % (16 * total / 1e9),
                      "parallelism": "replicas x%d (independent instances, no collective)" % world},
           "roofline": roof,
           "stages_ms_per_step": {k: round(v, 4) for k, v in sorted(stages.items())},
           "stage_pass_ms_per_step": stage_ms,
           "cpu_baseline": cpu,
           "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(16 * total),
                   "d2h_bytes_per_step": int(8 * total)},
           "gpu_launches": p.info()["launches_per_eval"] * steps, "clocks": clk, "steps": steps}
    if unbatched:
        res["unbatched"] = unbatched
        res["sigma_1.5"] = sigma15
        res["batching_speedup"] = unbatched["ms_per_step"] / ms_per_step
    p.close()
    del t, out
    torch.cuda.empty_cache()
    return res


def run_randstar(args, rank, world, local_rank, batch):
    dev = _setup(rank, world, local_rank)
    if rank == 0:
        from oracle import build as obuild
        obuild.build()
    r = randstar_arm(args, dev, local_rank, world, batch, args.steps, args.warmup)
    if rank != 0:
        return
    line = {"metric": r["metric"], "value": r["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": r["config"]}
    line.update({k: v for k, v in r.items() if k not in line and k not in ("metric", "steps")})
    print(json.dumps(line), flush=True)


def run_randstar_reference(args, rank, world, batch):
    from oracle import build as obuild
    obuild.build()
    if rank != 0:
        return
    if batch:
        problems, counts = W.random_star_batch()
        metric, name, streams = BATCH_METRIC, "randstar_batch32", [100 + i for i in range(32)]
    else:
        cfg = W.random_star()
        problems = [{"families": cfg["families"], "lam": cfg["lam"], "z": cfg["z"]}]
        counts, metric, name, streams = [100_000_000], R1000_METRIC, "randstar20_F1000", [1]
    sample = []
    for i, (m, st) in enumerate(zip(counts, streams)):
        x, y = W.square_targets(min(m, 4096), 1.2, 5, st)
        sample.append((x[: 4 if batch else 100], y[: 4 if batch else 100]))
    vals = []
    for _ in range(max(1, args.steps)):
        rate, cores, n_s, t_s, _ = _oracle_rate_t3(problems, sample, 8.0)
        vals.append(rate)
    v = statistics.median(vals)
    total = sum(counts)
    line = {"impl": "reference", "metric": metric, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / v * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "targets": total},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d targets, quadrature rebuilt + direct O(NM) FP64 sum, "
                                       "%.1f s per step" % (n_s, t_s)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ Koch snowflake (Sec. 4.3)
KOCH_METRIC = "Fresnel target pts/sec at 1e-6 rel L2 err (Koch snowflake L=13, 1000^2 grid)"
KOCH_LEVEL, KOCH_LZ = 13, 0.01


def _koch_oracle_rate(fams, budget_s):
    """The oracle as it stands (snowflake rule rebuilt + direct FP64 sum) on a
    bounded sample of the 1000^2 grid's targets; targets/s, and its values."""
    import oracle
    from oracle import direct
    xi, eta = oracle.grid_targets(1000, 1000, 0.003)
    rng = W.rng(13, 900)
    t0 = time.perf_counter()
    oracle.field(fams, KOCH_LZ, 1.0, xi[:16], eta[:16], output="occulter")   # calibration
    per = max((time.perf_counter() - t0) / 16, 1e-6)
    m = int(max(16, min(4096, budget_s / per)))
    idx = np.sort(rng.choice(len(xi), m, replace=False))
    t0 = time.perf_counter()
    u = oracle.field(fams, KOCH_LZ, 1.0, xi[idx], eta[idx], output="occulter")
    dt = time.perf_counter() - t0
    return m / dt, direct.max_threads(), m, dt, idx, u


def run_koch(args, rank, world, local_rank):
    """Sec. 4.3's snowflake: level 13 (67,108,864 triangles, p = 217 down to 1
    by level: 67.2M nodes regenerated every step), type 1 to the 1000^2 grid
    over [-1.5, 1.5)^2 at lz = 0.01, occulter field, FP32 fast mode."""
    import torch
    from paper_2010_05978_gb300 import Plan
    dev = _setup(rank, world, local_rank)
    fams = W.koch_families(KOCH_LEVEL, KOCH_LZ)
    n_tri = sum(len(f["tri"]) for f in fams)
    g = W.grid_spec(1000, 1000, 0.003)
    p, plan_ms = timed_plan(lambda: Plan(fams, KOCH_LZ, 1.0, TOL, precision="fp32", grid=g,
                                         output="occulter", recompute_nodes=True,
                                         sync_status=False))
    info = p.info()
    out = torch.empty((1000, 1000), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        p.eval(None, out)
    torch.cuda.synchronize()
    p.check()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    # the triangle list (3.2 GB) is larger than L2: no flush
    step_ms = time_steps(lambda: p.eval(None, out), stream, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    p.check()
    ms_per_step, value = aggregate_ranks(sum(step_ms), args.steps, 1e6, world, dev)
    u_dev = out.reshape(-1).clone()
    stages, stage_ms = stage_pass([("", p)], lambda: p.eval(None, out), stream, 3)
    h_out = torch.empty((1000, 1000), dtype=torch.complex64, pin_memory=True).numpy()
    e2e_ms = []
    for i in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.eval_host(None, h_out)
        torch.cuda.synchronize()
        if i:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    p.check()
    e2e = 1e6 * world / (statistics.median(e2e_ms) * 1e-3)
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    N, c64 = info["n_nodes"], 8
    nf = info["nf1"] * info["nf2"]
    ab = {"nodes_chirp_count": 48 * n_tri + 24 * N,   # triangle vertices in, records out
          "spread": 24 * N + nf * c64,
          "fft_rows": (nf + 1000 * info["nf2"]) * c64,
          "fft_cols_epilogue": (1000 * info["nf2"] + 1000 * 1000) * c64}
    roof = roofline("koch_L13", ab, stages, "stage pass: per-stage CUDA events, 3 steps; the "
                    "headline step is timed without stage events")
    rate, cores, n_s, t_s, idx, ref = _koch_oracle_rate(fams, 10.0)
    u = u_dev[torch.as_tensor(idx, device=dev)].cpu().numpy()
    err = dict(rel_error(u, ref, TOL, occulter=True), against="the oracle's direct FP64 sum "
               "(eq. faq) on its own snowflake rule, u^oc at sampled grid targets; outputs of the last timed step")
    line = {
        "metric": KOCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "koch_L13: Koch snowflake R=1 level 13 (%d triangles, p=%d..1 by "
                               "level), lz=0.01, u^oc on 1000x1000 grid h=0.003" % (
                                   n_tri, fams[0]["p"]),
                   "nodes": N, "triangles": n_tri, "targets": 1_000_000, "tol": TOL,
                   "precision": "fp32 spread/fft, double-float node coordinates and phases",
                   "nodes_recomputed_each_step": True,
                   "l2": "inputs larger than L2 (triangle list %.1f GB)" % (48 * n_tri / 1e9),
                   "parallelism": "replicas x%d (independent instances, no collective)" % world},
        "roofline": roof, "error": err, "plan_ms": plan_ms,
        "plan_plus_eval_ms": plan_ms + ms_per_step,
        "stages_ms_per_step": {k: round(v, 4) for k, v in sorted(stages.items())},
        "stage_pass_ms_per_step": stage_ms,
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d grid targets, snowflake rule rebuilt + direct O(NM) "
                                   "FP64 sum (eq. faq), %.1f s" % (n_s, t_s)},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(h_out.nbytes)},
        "gpu_launches": info["launches_per_eval"] * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_koch_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import build as obuild
    obuild.build()
    fams = W.koch_families(KOCH_LEVEL, KOCH_LZ)
    _koch_oracle_rate(fams, 1.0)
    vals, last = [], None
    for _ in range(max(1, args.steps)):
        last = _koch_oracle_rate(fams, 8.0)
        vals.append(last[0])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": KOCH_METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e6 / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "koch_L13", "targets": 1_000_000},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last[1], "kind": "oracle",
                             "sample": "%d grid targets per step, snowflake rule rebuilt + direct "
                                       "O(NM) FP64 sum, %.1f s" % (last[2], last[3])},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="star5_F100",
                    choices=["star5_F100", "starshade_sweep", "randstar_F1000", "randstar_batch32",
                             "koch_L13"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="star5_F100 only: fp64 times the plain FP64 path at the same "
                         "tolerance (1e-6), for comparison with the FP32 fast mode")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="star5_F100 only: time the headline workload alone (no FP64 path, "
                         "sweep or F=1000 objects in the line)")
    ap.add_argument("--deterministic", action="store_true",
                    help="star5_F100 only: plans in deterministic mode (exact fixed-point "
                         "spreading, bitwise-repeatable outputs); the line carries the star alone")
    ap.add_argument("--targets", type=int, default=0,
                    help="randstar_F1000 only: scattered targets (default 1e8; fewer for small "
                         "profiling captures)")
    ap.add_argument("--lambdas", type=int, default=64,
                    help="starshade_sweep only: wavelengths per sweep (64 is the benchmark; "
                         "fewer for small profiling captures)")
    args = ap.parse_args()
    if args.precision != "fp32" and args.workload != "star5_F100":
        ap.error("--precision fp64 is offered for the star5_F100 workload only")
    if args.deterministic and args.workload != "star5_F100":
        ap.error("--deterministic is offered for the star5_F100 workload only")
    sweep = args.workload == "starshade_sweep"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload == "koch_L13":
            run_koch_reference(args, rank, world)
        elif args.workload in ("randstar_F1000", "randstar_batch32"):
            run_randstar_reference(args, rank, world, args.workload == "randstar_batch32")
        else:
            (run_sweep_reference if sweep else run_reference)(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "koch_L13":
        run_koch(args, rank, world, local_rank)
    elif args.workload in ("randstar_F1000", "randstar_batch32"):
        run_randstar(args, rank, world, local_rank, args.workload == "randstar_batch32")
    else:
        (run_sweep if sweep else run_ours)(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
