#!/usr/bin/env python
"""Benchmark of the fast multivariate ECDF / Laplacian KDE hot path on GB300.

One step is one pass of the whole hot path over the d=3, N=1e6 workload
(correlated Gaussian, S_ij = 0.5, FP32 inputs):

  * ecdf_grid   -- binning + histogram + orthant scans on a 256^3 grid, all
                   8 orthants, exact int64 counts (Sec. 2.1);
  * ecdf_points -- rank transform + divide-and-conquer, all 8 orthants at the
                   N sample points, exact counts (Sec. 2.2, Appendix D);
  * kde_laplace -- Laplacian KDE at the N sample points, h = 0.1, mixed
                   precision (Sec. 3.1).

value = N sample points / step time (each point gets its 8 orthant counts and
its density; the 256^3 grid is evaluated alongside).  The three calls are
independent and run on three streams (--serial: one after another; the
per-call times are reported beside the step either way).  Inputs are resident in
HBM; L2 (129 MB) is flushed by writing a 256 MB buffer between timed steps.
`e2e` times the same step through the C ABI with pinned HOST buffers (copies
in and out inside the timed region).  `--impl reference` times the CPU oracle
on a bounded sample of the same workload.

With --gpus N (torchrun) every rank runs an independent replica (the
single-dataset sample-point problem couples every pair of points and does not
shard); value aggregates all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ECDF/Laplace-KDE points/sec at N=1e6 vs FP64 GPU path; % HBM roofline"
UNIT = "points/s"
N_POINTS = 1_000_000
D = 3
M_AXIS = 256
H = 0.1
WORKLOAD = "ecdf_gauss3_d3_n1e6_grid256_kde_h0.1"
# sizes of the d = 5, 6 rows of the runtime-versus-N study (the sweep has 16
# and 32 channels there; the paper's Tables 2 and 4 go to N = 1.28e6 at d = 6)
SCALING_HIGH_D = {5: (10_000, 30_000, 100_000, 300_000), 6: (10_000, 30_000, 100_000)}


def _args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--serial", action="store_true",
                    help="run the step's three calls one after another on one stream")
    ap.add_argument("--scaling", action="store_true",
                    help="time the sample-point counts, the KDE and the grid counts over d and N (the "
                         "paper's runtime-versus-N study) and print one JSON line")
    ap.add_argument("--no-c5", action="store_true", help="skip the d=4, N=4e6 leave-one-out workload")
    ap.add_argument("--no-c5-search", action="store_true", help="skip its 20-step bandwidth search")
    ap.add_argument("--no-scaling", action="store_true", help="skip the d = 5, 6 runtime-versus-N rows")
    ap.add_argument("--only", default=None, choices=["grid", "points", "kde", "kde64", "kreg"],
                    help="run one operation per step (profiling of a single kernel family)")
    return ap.parse_args(argv)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Families whose work is counted in floating-point operations (the tile-local
# kernel-sum sweep is bound by instruction issue, not by HBM); they are held
# against the FP32 lane peak: SMs (read from the device) x 128 FP32 lanes x
# the maximum SM clock (the sampled clocks.max.sm, else the measured-peaks
# file, else 2070 MHz), one non-fused operation per lane and clock.
ALU_FAMILIES = ("kernel_local",)


def fp32_peak(sms, max_mhz, clock_source):
    """(TFLOP/s, description) of the FP32 lane peak."""
    return (sms * 128 * max_mhz * 1e6 / 1e12,
            "derived: %d SMs (device properties) x 128 FP32 lanes x %.0f MHz max SM clock (%s)"
            % (sms, max_mhz, clock_source))


def _max_sm_mhz(clk):
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"]), "nvidia-smi clocks.max.sm"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json"
    except Exception:
        return 2070.0, "nominal"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region.

    start() launches the sampler and waits (at most `ready_s`) for its first
    line, so that it is running before the region opens; begin() and stop()
    bracket the region, and only the lines that arrive inside it (plus
    `grace_s` for the sample in flight when it closes) are summarised.  When
    the region is shorter than the sampling period and no line falls inside,
    the first line after begin() stands for it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index, period_ms=200, cmd=None, ready_s=5.0, grace_s=0.05):
        self.index = index
        self.period_s = period_ms / 1e3
        self.cmd = cmd or ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                           "--format=csv,noheader,nounits", "-lms", str(period_ms)]
        self.ready_s = ready_s
        self.grace_s = grace_s
        self.proc = None
        self.lines = []            # (arrival time, line)
        self.thread = None
        self.first = threading.Event()
        self.t_begin = None
        self.t_end = None

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        self.first.wait(timeout=self.ready_s)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))
            self.first.set()

    def begin(self):
        self.t_begin = time.perf_counter()

    def stop(self):
        self.t_end = time.perf_counter()
        if not self.proc:
            return None
        if self.t_begin is None:
            self.t_begin = self.t_end
        # let the line of a sample taken just before the region closed arrive;
        # a region shorter than the period waits (at most two periods) for the
        # first sample after it opened
        time.sleep(self.grace_s)
        deadline = time.perf_counter() + 2.0 * self.period_s
        while time.perf_counter() < deadline and not any(t >= self.t_begin for t, _ in list(self.lines)):
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()

    @classmethod
    def parse(cls, line):
        """(sm MHz, max sm MHz, set of active reasons) of one CSV line, or None."""
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            return None
        try:
            sm, mx = float(parts[1]), float(parts[2])
        except ValueError:
            return None
        active = {nm for nm, v in zip(cls.REASONS, parts[5:9]) if v.lower().startswith("active")}
        return sm, mx, active

    def summary(self):
        parsed = [(t, self.parse(ln)) for t, ln in self.lines]
        parsed = [(t, p) for t, p in parsed if p is not None]
        inside = [p for t, p in parsed if self.t_begin <= t <= self.t_end + self.grace_s]
        if not inside:
            inside = [p for t, p in parsed if t >= self.t_begin][:1]
        if not inside:
            return None
        reasons = set()
        for p in inside:
            reasons |= p[2]
        return {"sm_mhz": statistics.median(p[0] for p in inside), "sm_max_mhz": max(p[1] for p in inside),
                "reasons": sorted(reasons), "samples": len(inside)}


def _workload(n):
    from paper_2005_03246_gb300 import datagen
    data = datagen.ecdf_gauss3(n=n)
    return data["x"], data["grid"]


# ----------------------------------------------------------------------------- CPU oracle


def _oracle_sample(x, grid, s, seed=0, keep=False):
    """The oracle on s sample points: their orthant counts and density, plus
    s * (grid points / N) random grid points' orthant counts.  Returns the
    seconds taken, and with ``keep`` also the sample and the oracle's values."""
    import oracle
    from paper_2005_03246_gb300 import datagen
    n = x.shape[0]
    dim = len(grid)
    m = [len(a) for a in grid]
    idx = datagen.sample_targets(n, s, seed=seed)
    r = np.random.default_rng(seed)
    gcount = max(1, int(round(s * float(np.prod(m)) / n)))
    gi = np.stack([r.integers(0, m[k], size=gcount) for k in range(dim)], axis=1)
    gz = np.stack([grid[k][gi[:, k]] for k in range(dim)], axis=1)
    t0 = time.perf_counter()
    points = oracle.orthant_sums(x, z=x[idx])
    kde = oracle.kde_laplace(x, H, z=x[idx])
    gcounts = oracle.orthant_sums(x, z=gz)
    t = time.perf_counter() - t0
    if not keep:
        return t
    return t, {"idx": idx, "gi": gi, "points": points, "kde": kde, "grid": gcounts}


def _gather(g, p, f, ref):
    """The step's GPU outputs (grid counts [2^d, M_1..M_d], sample-point counts
    [2^d, N], densities [N]) at the oracle's sample, as host arrays."""
    import torch
    # host-side bounds checks: no index reaches the device unless it is in range
    dim = ref["gi"].shape[1]
    if (p.dim() != 2 or f.dim() != 1 or g.dim() != dim + 1 or g.shape[0] != p.shape[0]
            or int(ref["idx"].max()) >= min(p.shape[1], f.shape[0]) or int(ref["idx"].min()) < 0
            or any(int(ref["gi"][:, k].max()) >= g.shape[k + 1] for k in range(dim)) or int(ref["gi"].min()) < 0):
        raise ValueError("outputs of shapes %s, %s, %s do not cover the sample"
                         % (tuple(g.shape), tuple(p.shape), tuple(f.shape)))
    idx = torch.as_tensor(ref["idx"], device=p.device)
    gi = [torch.as_tensor(ref["gi"][:, k], device=g.device) for k in range(dim)]
    return {"points": p[:, idx].cpu().numpy(), "kde": f[idx.to(f.device)].cpu().numpy(),
            "grid": g[(slice(None), *gi)].cpu().numpy()}


def _accuracy(ref, got, kde_tol=1e-5):
    """Agreement of the GPU outputs with the oracle on the sample: count
    mismatches (counts are exact, so any is an error) and the mixed-path KDE's
    largest relative error on values >= 1e-6 of the sample's largest."""
    fr = np.asarray(ref["kde"], dtype=np.float64)
    fg = np.asarray(got["kde"], dtype=np.float64)
    sel = fr >= 1e-6 * fr.max() if fr.size else np.zeros(0, dtype=bool)
    rel = float((np.abs(fg[sel] - fr[sel]) / fr[sel]).max()) if sel.any() else 0.0
    return {"reference": "oracle (brute force, FP64 / exact int64) on the cpu_baseline sample",
            "sample_points": int(len(ref["idx"])), "grid_points": int(ref["gi"].shape[0]),
            "points_count_mismatches": int(np.count_nonzero(ref["points"] != got["points"])),
            "grid_count_mismatches": int(np.count_nonzero(ref["grid"] != got["grid"])),
            "kde_mixed_max_rel_err": rel, "kde_tolerance": kde_tol}


def _rel_pos(got, ref):
    """Largest relative error on entries >= 1e-6 of the largest reference."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sel = np.abs(ref) >= 1e-6 * np.abs(ref).max() if ref.size else np.zeros(0, dtype=bool)
    return float((np.abs(got[sel] - ref[sel]) / np.abs(ref[sel])).max()) if sel.any() else 0.0


def _rel_cond(got, ref, cond):
    """Error of signed results relative to their condition (the same quantity
    computed from magnitudes), with the scale floored at 1e-6 of the largest
    reference value."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.maximum(np.abs(np.asarray(cond, dtype=np.float64)), 1e-6 * np.abs(ref).max())
    return float((np.abs(got - ref) / scale).max()) if ref.size else 0.0


def _c9(got, ref):
    """|g - o| / max(|o|, 1e-6 max|o|) over every entry."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float((np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())).max()) if ref.size else 0.0


def _accuracy_extras(samples, x_step):
    """The oracle's error for every other result the bench times: the batched
    outputs, the adjoint, the d=2 copula KDE / Nadaraya-Watson / adjoint, the
    weighted d=3 sums and the d=4 leave-one-out densities."""
    import oracle
    acc = {}
    if "batched_mixed" in samples:
        for path in ("mixed", "fp64"):
            cm, ke, kc = 0, 0.0, 0.0
            for xb, yb, e, k in samples["batched_" + path]:
                cm += int(np.count_nonzero(oracle.orthant_sums(xb) != e))
                ref = oracle.kde_laplace(xb, H, w=yb)
                cond = oracle.kde_laplace(xb, H, w=np.abs(yb))
                ke = max(ke, _rel_cond(k, ref, cond))
                kc = max(kc, _c9(k, ref))
            acc["batched_" + path] = {"datasets_checked": len(samples["batched_" + path]),
                                      "count_mismatches": cm, "kde_err_rel_to_abs_weights": ke, "kde_c9": kc}
    if "backward_d3" in samples:
        b = samples["backward_d3"]
        ref = oracle.kde_laplace(x_step, H, z=x_step[b["idx"]])
        acc["kde_backward_d3_grad_w"] = {"targets": len(b["idx"]), "max_rel_err": _rel_pos(b["grad_w"], ref)}
    if "c3" in samples:
        c = samples["c3"]
        xs, ys, idx = c["x"], c["y"], c["idx"]
        z = xs[idx]
        rows = {}
        for (h, path), (f, m) in c["values"].items():
            rf = oracle.kde_laplace(xs, h, z=z)
            rm = oracle.kreg_laplace(xs, ys, h, z=z)
            cm = oracle.kreg_laplace(xs, np.abs(ys), h, z=z)
            rows["h%g_%s" % (h, path)] = {"kde_max_rel_err": _rel_pos(f, rf), "nw_err_rel_to_abs_y": _rel_cond(m, rm, cm),
                                          "nw_c9": _c9(m, rm)}
        a = c["adjoint"]
        rw, rz, rh = oracle.kde_grad(xs, a["h"], a["g"], z=a["z"])
        for path in ("mixed", "fp64"):
            sw, gw, gz, gh = a[path]
            rows["adjoint_%s" % path] = {
                "grad_w_err_rel_max": float(np.abs(gw - rw[sw]).max() / np.abs(rw).max()),
                "grad_z_err_rel_max": float(np.abs(gz - rz).max() / np.abs(rz).max()),
                "grad_h_err_rel_max": float(np.abs(gh - rh).max() / np.abs(rh).max())}
        rows["targets"] = len(idx)
        acc["c3_copula_d2"] = rows
    if "c2w" in samples:
        c = samples["c2w"]
        ref = oracle.orthant_sums(x_step, y=c["y"], z=x_step[c["idx"]])
        acc["c2_weighted_d3"] = {"targets": len(c["idx"]), **{
            "%s_max_rel_err" % path: _rel_pos(c[path], ref) for path in ("mixed", "fp64")}}
    if "c5" in samples:
        c = samples["c5"]
        ref = oracle.kde_at_points(c["x"], c["h"], c["idx"], loo=True)
        acc["c5_loo_d4"] = {"targets": len(c["idx"]), **{
            "%s_loo_density_max_rel_err" % path: _rel_pos(c[path], ref) for path in ("mixed", "fp64")}}
    return acc


def _cpu_baseline(x, grid, target_s=15.0, gpu_out=None, extra_samples=None):
    """The oracle timed on a bounded sample of the workload.  With the step's
    GPU outputs (g, p, f, f64) it also reports their agreement with the
    oracle's values on that sample (``accuracy``), and with the samples of the
    other workloads their errors too."""
    import oracle
    oracle.build()
    n = x.shape[0]
    gcount = lambda s: max(1, int(round(s * float(np.prod([len(a) for a in grid])) / n)))
    s = 16
    t = _oracle_sample(x, grid, s)
    s = int(max(16, min(4096, s * target_s / max(t, 1e-3) * 0.8)))
    t, ref = _oracle_sample(x, grid, s, seed=1, keep=True)
    out = {"value": s / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
           "sample": "%d of the %d sample points (%d orthant counts + density each, h=%g) and %d "
                     "random grid points (%d orthant counts each), all against the full N sources; "
                     "%.1f s" % (s, n, 1 << len(grid), H, gcount(s), 1 << len(grid), t)}
    if gpu_out is not None:
        try:
            g, p, f, f64 = gpu_out
            out["accuracy"] = _accuracy(ref, _gather(g, p, f, ref))
            out["accuracy"]["kde_fp64_max_rel_err"] = _rel_pos(_gather(g, p, f64, ref)["kde"], ref["kde"])
        except Exception as e:   # the check must not cost the bench line
            out["accuracy"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if extra_samples:
        try:
            out.setdefault("accuracy", {})["other_workloads"] = _accuracy_extras(extra_samples, x)
        except Exception as e:
            out.setdefault("accuracy", {})["other_workloads"] = {"error": "%s: %s" % (type(e).__name__, e)}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    x, grid = _workload(args.n)
    # each step: a bounded sample of oracle work, sized so that the warm-up and
    # timed steps together take about 90 s (between 0.3 and 3 s per step)
    per_step = min(3.0, max(0.3, 90.0 / max(1, args.steps + args.warmup)))
    s = 16
    t = _oracle_sample(x, grid, s)
    s = int(max(16, min(4096, s * per_step / max(t, 1e-3))))
    for w in range(args.warmup):
        _oracle_sample(x, grid, s, seed=100 + w)
    times = [_oracle_sample(x, grid, s, seed=200 + k) for k in range(args.steps)]
    tm = sum(times) / len(times)
    value = s / tm
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tm * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n": args.n, "d": D, "grid": [M_AXIS] * D, "h": H,
                       "sample_points_per_step": s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "%d sample points + %d grid points per step against all N sources"
                                       % (s, max(1, int(round(s * M_AXIS ** D / args.n))))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm


def aggregate_replicas(total_ms, steps, n, ws, device="cpu"):
    """Whole-job throughput of `ws` independent replicas, each timing `steps`
    steps of `n` points in `total_ms`: the step time is the slowest rank's
    (all-reduce MAX over the process group when ws > 1) and the value counts
    the points of all ranks.  Returns (ms_per_step, points per second)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_step = float(t.item()) / steps
    return ms_step, ws * n / (ms_step / 1e3)


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2005_03246_gb300 as fk
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()

    x_np, grid = _workload(args.n)
    n = x_np.shape[0]
    x = torch.as_tensor(x_np, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    ywt = torch.as_tensor(np.sin(x_np.astype(np.float64).sum(axis=1)).astype(np.float32), device=dev)
    only = {"grid": lambda: fk.ecdf_grid(x, grid), "points": lambda: fk.ecdf_points(x),
            "kde": lambda: fk.kde_laplace(x, H, path="mixed"),
            "kde64": lambda: fk.kde_laplace(x, H, path="fp64"),
            "kreg": lambda: fk.kreg_laplace(x, ywt, H, path="mixed")}

    # The three calls of a step are independent: unless --serial, the KDE and
    # the grid counts run on their own streams (forked from and joined back to
    # the timing stream by events) while the sample-point counts run on the
    # timing stream; they are issued last because they read their tie
    # statistics back once.
    side = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

    def step(kde_path="mixed"):
        if args.only:
            return only[args.only]()
        if args.serial:
            g = fk.ecdf_grid(x, grid)
            p = fk.ecdf_points(x)
            f = fk.kde_laplace(x, H, path=kde_path)
            return g, p, f
        fork = torch.cuda.Event()
        fork.record(stream)
        for s in side:
            s.wait_event(fork)
        with torch.cuda.stream(side[0]):
            f = fk.kde_laplace(x, H, path=kde_path)
        with torch.cuda.stream(side[1]):
            g = fk.ecdf_grid(x, grid)
        p = fk.ecdf_points(x)
        for s in side:
            join = torch.cuda.Event()
            join.record(s)
            stream.wait_event(join)
        return g, p, f

    for _ in range(max(3, args.warmup)):
        out = step()
    del out
    torch.cuda.synchronize()

    # ---- timed region (device time, CUDA events on the launching stream)
    clocks = ClockSampler(local)
    clocks.start()
    lib.fk_profile_reset()
    lib.fk_profile_enable(1)
    l0 = lib.fk_kernel_launches()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        del out
    torch.cuda.synchronize()
    launches = lib.fk_kernel_launches() - l0
    lib.fk_profile_enable(0)
    clk = clocks.stop()
    total_ms = float(sum(times))
    ms_step, value = aggregate_replicas(total_ms, args.steps, n, ws, dev)

    # ---- roofline of the dominant kernel family
    fams = {}
    for name, fid in _lib.PROFILE_FAMILIES.items():
        tot = ctypes.c_double(0)
        cnt = ctypes.c_uint64(0)
        by = ctypes.c_double(0)
        lib.fk_profile_read(fid, ctypes.byref(tot), ctypes.byref(cnt), ctypes.byref(by))
        if cnt.value:
            busy = ctypes.c_double(0)
            lib.fk_profile_busy(fid, ctypes.byref(busy))
            fams[name] = (tot.value, cnt.value, by.value, busy.value)
    lib.fk_profile_reset()
    peak, peak_kind = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE = fp32_peak(sms, *_max_sm_mhz(clk))
    dom = max(fams.items(), key=lambda kv: kv[1][3]) if fams else None
    roofline = None
    if dom:
        name, (tms, cnt, by, busy) = dom
        per_launch_s = (tms / cnt) / 1e3
        if name in ALU_FAMILIES:
            # arithmetic-bound family: work = floating-point operations
            roofline = {"bound": "alu", "kernel": name, "achieved": (by / cnt) / per_launch_s / 1e12,
                        "peak": FP32_PEAK_TFLOPS, "peak_source": FP32_PEAK_SOURCE, "unit": "TFLOP/s"}
            roofline["frac"] = roofline["achieved"] / FP32_PEAK_TFLOPS
            roofline["alg_flop_per_launch"] = by / cnt
        else:
            roofline = {"bound": "hbm", "kernel": name, "achieved": (by / cnt) / per_launch_s / 1e9,
                        "peak": peak, "peak_source": peak_kind, "unit": "GB/s"}
            roofline["frac"] = roofline["achieved"] / peak
            roofline["alg_bytes_per_launch"] = by / cnt
        # The engines run independent sorts on concurrent streams, so launch
        # durations overlap: the per-launch figure above counts a launch's
        # whole interval, while the busy figure divides the family's work by
        # the union of its launch intervals.
        scale = 1e12 if name in ALU_FAMILIES else 1e9
        roofline["achieved_busy"] = by / (busy / 1e3) / scale if busy > 0 else None
        roofline["frac_busy"] = (roofline["achieved_busy"] / roofline["peak"]) if busy > 0 else None
        roofline.update({"traffic": _traffic(name, by / cnt), "launches": cnt,
                         "avg_launch_us": tms / cnt * 1e3, "busy_ms_per_step": busy / args.steps,
                         "share_of_step": busy / total_ms})

    # compulsory I/O of a step (read x once per call, write every output once)
    # over the step time: the floor any implementation of the step must move
    gpts = M_AXIS ** D
    b_io = 3 * x_np.nbytes + 8 * gpts * 8 + 8 * n * 8 + n * 8
    io_floor = {"bytes_per_step": int(b_io), "gbs": b_io / (ms_step / 1e3) / 1e9,
                "frac_of_peak": b_io / (ms_step / 1e3) / 1e9 / peak}

    def _rate(name, v):   # work per busy second
        if v[3] <= 0:
            return None
        return v[2] / (v[3] / 1e3) / (1e12 if name in ALU_FAMILIES else 1e9)

    breakdown = {k: {"ms_per_step": v[0] / args.steps, "busy_ms_per_step": v[3] / args.steps,
                     "launches_per_step": v[1] / args.steps,
                     "rate": _rate(k, v), "rate_unit": "TFLOP/s" if k in ALU_FAMILIES else "GB/s"}
                 for k, v in fams.items()}

    # ---- per-call split and the FP64 GPU path on the same inputs
    def timed(fn, reps=3):
        vals = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            b.synchronize()
            vals.append(a.elapsed_time(b))
            del r
        return statistics.median(vals)

    if args.only:
        print(json.dumps({"only": args.only, "n": n, "ms_per_step": ms_step, "families": breakdown}), flush=True)
        return 0
    split = {"ecdf_grid_ms": timed(lambda: fk.ecdf_grid(x, grid)),
             "ecdf_points_ms": timed(lambda: fk.ecdf_points(x)),
             "kde_mixed_ms": timed(lambda: fk.kde_laplace(x, H, path="mixed"))}
    kde64 = timed(lambda: fk.kde_laplace(x, H, path="fp64"))
    fp64 = {"kde_fp64_ms": kde64, "kde_mixed_ms": split["kde_mixed_ms"],
            "mixed_speedup": kde64 / split["kde_mixed_ms"]}

    # ---- roofline of each call: the algorithmic bytes of all its profiled
    # passes (each pass reading its inputs once and writing its outputs once,
    # as the library records them) over the call's own time
    def call_bytes(fn):
        lib.fk_profile_reset()
        lib.fk_profile_enable(1)
        r = fn()
        torch.cuda.synchronize()
        lib.fk_profile_enable(0)
        tot = 0.0
        for fid in _lib.PROFILE_FAMILIES.values():
            b = ctypes.c_double(0)
            lib.fk_profile_read_bytes(fid, ctypes.byref(b))
            tot += b.value
        lib.fk_profile_reset()
        del r
        return tot

    per_call = {}
    for key, fn, ms in (("ecdf_points", lambda: fk.ecdf_points(x), split["ecdf_points_ms"]),
                        ("kde_laplace_mixed", lambda: fk.kde_laplace(x, H, path="mixed"), split["kde_mixed_ms"]),
                        ("kde_laplace_fp64", lambda: fk.kde_laplace(x, H, path="fp64"), kde64),
                        ("ecdf_grid", lambda: fk.ecdf_grid(x, grid), split["ecdf_grid_ms"])):
        b = call_bytes(fn)
        a = b / (ms / 1e3) / 1e9
        per_call[key] = {"alg_bytes": b, "ms": ms, "achieved": a, "unit": "GB/s", "peak": peak,
                         "peak_source": peak_kind, "frac": a / peak}

    # ---- the same step with the KDE on the all-FP64 path (the paper's precision)
    fp64_step = None
    if not args.only:
        def step64():
            return step(kde_path="fp64")
        for _ in range(2):
            r = step64()
        del r
        torch.cuda.synchronize()
        t64 = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = step64()
            b.record(stream)
            b.synchronize()
            t64.append(a.elapsed_time(b))
            del r
        ms64 = float(sum(t64)) / len(t64)
        ms64, v64 = aggregate_replicas(ms64 * len(t64), len(t64), n, ws, dev)
        fp64_step = {"ms_per_step": ms64, "value": v64, "unit": UNIT, "steps": len(t64),
                     "dtype": "u32/i64 counts; f64 KDE", "mixed_over_fp64": value / v64}

    # ---- other hot-path rows on their own workloads (reported beside the step)
    extras = {}
    samples = {}
    if not args.no_extras:
        extras, samples = _extras(fk, torch, dev, x, stream, flush, timed, args)

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(lib, x_np, grid, args, dev)
        # whole job: the slowest rank's step time, the points of all ranks
        ms_e2e, e2e["value"] = aggregate_replicas(e2e["ms_per_step"], 1, n, ws, dev)
        e2e["ms_per_step"] = ms_e2e

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        # one more (untimed) step whose outputs are checked against the
        # oracle's values on the CPU sample
        try:
            outs = tuple(step()) + (fk.kde_laplace(x, H, path="fp64"),)
            torch.cuda.synchronize()
        except Exception:
            outs = None
        cpu = _cpu_baseline(x_np, grid, gpu_out=outs, extra_samples=samples)
        del outs

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32/i64 counts; f32+f64 (mixed KDE)", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "d": D, "grid": [M_AXIS] * D, "orthants": 8,
                           "h": H, "kde_path": "mixed", "l2": "flushed (256 MB write) between steps",
                           "calls": "one after another" if args.serial else
                                    "independent calls on three streams (KDE, grid counts, sample-point counts)",
                           "parallelism": "replicas" if ws > 1 else "single"},
                "gpu_launches": int(launches), "roofline": roofline, "roofline_per_call": per_call,
                "io_floor": io_floor, "kernel_families": breakdown,
                "split": split, "fp64_path": fp64, "fp64_step": fp64_step, "extras": extras, "e2e": e2e,
                "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _extras(fk, torch, dev, x, stream, flush, timed, args):
    """The other hot-path workloads, timed beside the step (ms, CUDA events,
    L2 flushed): the 512-dataset batch (graph replay; mixed vs FP64), the KDE
    adjoint at N=1e6, d=3, the d=2 copula workload (KDE and Nadaraya-Watson at
    three bandwidths, both paths, and the adjoint), the weighted d=3 orthant
    sums, the d=4 leave-one-out likelihood and bandwidth search, the grid KDE
    study and the other estimators.  Returns (timings, samples): `samples`
    holds GPU outputs at seeded indices, which the cpu_baseline leg compares
    with the oracle."""
    from paper_2005_03246_gb300 import datagen
    out, samples = {}, {}
    sets = datagen.batched()
    xs = [torch.as_tensor(s["x"], device=dev) for s in sets]
    ys = [torch.as_tensor(s["y"], device=dev) for s in sets]
    pts = int(sum(s["n"] for s in sets))
    # each path with the configuration its autotuner picks (and the default one)
    bm = fk.Batched(xs, ys, h=H, path="mixed", graph=True, config="tune")
    bd = fk.Batched(xs, ys, h=H, path="fp64", graph=True, config="tune")
    bm0 = fk.Batched(xs, ys, h=H, path="mixed", graph=True)
    tm = timed(lambda: bm.run(), reps=5)
    td = timed(lambda: bd.run(), reps=5)
    tm0 = timed(lambda: bm0.run(), reps=5)
    out["batched"] = {"workload": "512 datasets, N log-uniform [1e3,1e5], d 2/3, U[0,1] FP32; all orthant "
                                  "counts + Laplacian KDE h=0.1 weighted by y; CUDA-graph replay",
                      "points": pts, "mixed_ms": tm, "fp64_ms": td, "points_per_s": pts / (tm / 1e3),
                      "mixed_speedup": td / tm, "mixed_config": bm.config, "fp64_config": bd.config,
                      "mixed_default_config_ms": tm0}
    # outputs of six datasets (three of each dimension, the smallest first) for the oracle
    chk = sorted(range(len(sets)), key=lambda b: sets[b]["n"])
    chk = [b for b in chk if sets[b]["d"] == 2][:3] + [b for b in chk if sets[b]["d"] == 3][:3]
    for name, bb in (("mixed", bm), ("fp64", bd)):
        e, k = bb.run()
        torch.cuda.synchronize()
        samples["batched_" + name] = [(sets[b]["x"], sets[b]["y"], e[b].cpu().numpy(), k[b].cpu().numpy())
                                      for b in chk]
    del bm, bd, bm0
    # KDE adjoint (grad w, grad h) at N=1e6, d=3, upstream gradient 1: grad_w[i]
    # is the unweighted kernel sum at x_i (the kernel is symmetric)
    g = torch.ones(x.shape[0], dtype=torch.float64, device=dev)
    out["kde_backward_ms"] = timed(lambda: fk.kde_laplace_backward(x, H, g, need_w=True, need_z=False,
                                                                   need_h=True, path="mixed"), reps=3)
    gw, _, gh = fk.kde_laplace_backward(x, H, g, need_w=True, need_z=False, need_h=True, path="mixed")
    idx = datagen.sample_targets(x.shape[0], 128, seed=77)
    samples["backward_d3"] = {"idx": idx, "grad_w": gw[torch.as_tensor(idx, device=dev)].cpu().numpy()}
    del gw, gh
    out["c3_copula_d2"] = _c3(fk, torch, dev, timed, samples)
    out["c2_weighted_d3"] = _c2_weighted(fk, torch, dev, x, timed, samples)
    if not args.no_c5:
        out["c5_loo_d4"] = _c5(fk, torch, dev, timed, samples, search=not args.no_c5_search)
    out["kde_grid"] = _grid_kde_study(fk, torch, x, timed)
    out["other_estimators"] = _other_estimators(fk, torch, x, timed)
    if not args.no_scaling:
        out["scaling_high_d"] = {
            "data": "correlated Gaussian S_ij = 0.5, FP32; all 2^d orthant counts and the mixed KDE (h = 0.1) "
                    "at the sample points; ms and ns / (N log2^(d-1) N)",
            "rows": _scaling_rows(fk, torch, dev, [(5, SCALING_HIGH_D[5][:3]), (6, SCALING_HIGH_D[6][:3])],
                                  lambda fn, reps: timed(lambda: fn(), reps=reps), grid=False, reps=2)}
    return out, samples


def _c3(fk, torch, dev, timed, samples):
    """d=2 Gaussian copula with Student-t4 marginals, N=1e6: KDE and
    Nadaraya-Watson at the sample points for h in {0.05, 0.1, 0.3}, mixed and
    FP64 paths; the adjoint (grad w, z, h) at 4096 explicit targets."""
    from paper_2005_03246_gb300 import datagen
    d = datagen.copula_t4()
    xn, yn = d["x"], d["y"]
    x = torch.as_tensor(xn, device=dev)
    y = torch.as_tensor(yn, device=dev)
    n = xn.shape[0]
    idx = datagen.sample_targets(n, 256, seed=31)
    it = torch.as_tensor(idx, device=dev)
    res = {"workload": "d=2 Gaussian copula rho=0.7, t4 marginals, N=1e6, FP32; y = sin(x1+x2) + 0.1 N(0,1)"}
    smp = {"x": xn, "y": yn, "idx": idx, "values": {}}
    for h in (0.05, 0.1, 0.3):
        row = {}
        for path in ("mixed", "fp64"):
            row["kde_%s_ms" % path] = timed(lambda: fk.kde_laplace(x, h, path=path), reps=3)
            row["nw_%s_ms" % path] = timed(lambda: fk.kreg_laplace(x, y, h, path=path), reps=3)
            f = fk.kde_laplace(x, h, path=path)
            m = fk.kreg_laplace(x, y, h, path=path)
            smp["values"][(h, path)] = (f[it].cpu().numpy(), m[it].cpu().numpy())
            del f, m
        row["kde_mixed_speedup"] = row["kde_fp64_ms"] / row["kde_mixed_ms"]
        row["nw_mixed_speedup"] = row["nw_fp64_ms"] / row["nw_mixed_ms"]
        row["kde_points_per_s_mixed"] = n / (row["kde_mixed_ms"] / 1e3)
        res["h%g" % h] = row
    r = np.random.default_rng(33)
    m = 4096
    zn = (xn[r.choice(n, m, replace=False)] + r.normal(0.0, 0.05, (m, 2))).astype(np.float32)
    gn = r.standard_normal(m)
    z = torch.as_tensor(zn, device=dev)
    g = torch.as_tensor(gn, device=dev)
    hv = np.array([0.1, 0.12])
    adj = {"targets": m, "h": hv.tolist()}
    for path in ("mixed", "fp64"):
        adj["%s_ms" % path] = timed(lambda: fk.kde_laplace_backward(x, hv, g, z=z, path=path), reps=3)
    adj["mixed_speedup"] = adj["fp64_ms"] / adj["mixed_ms"]
    res["adjoint"] = adj
    # a 512-target slice of the same adjoint for the oracle
    zs, gs = zn[:512], gn[:512]
    smp["adjoint"] = {"z": zs, "g": gs, "h": hv}
    for path in ("mixed", "fp64"):
        gw, gz, gh = fk.kde_laplace_backward(x, hv, torch.as_tensor(gs, device=dev),
                                             z=torch.as_tensor(zs, device=dev), path=path)
        sw = datagen.sample_targets(n, 128, seed=34)
        smp["adjoint"][path] = (sw, gw[torch.as_tensor(sw, device=dev)].cpu().numpy(), gz.cpu().numpy(),
                                gh.cpu().numpy())
    samples["c3"] = smp
    return res


def _c2_weighted(fk, torch, dev, x, timed, samples):
    """All 8 weighted orthant sums at the N=1e6 sample points of the d=3
    workload, y ~ U[0,1], both paths."""
    from paper_2005_03246_gb300 import datagen
    d = datagen.ecdf_gauss3()
    yn = d["y"]
    y = torch.as_tensor(yn, device=dev)
    idx = datagen.sample_targets(x.shape[0], 128, seed=21)
    it = torch.as_tensor(idx, device=dev)
    res = {"workload": "d=3 correlated Gaussian N=1e6, y ~ U[0,1], all 8 orthants at the sample points"}
    smp = {"y": yn, "idx": idx}
    for path in ("mixed", "fp64"):
        res["%s_ms" % path] = timed(lambda: fk.ecdf_points(x, y=y, path=path), reps=3)
        o = fk.ecdf_points(x, y=y, path=path)
        smp[path] = o[:, it].cpu().numpy()
        del o
    res["mixed_speedup"] = res["fp64_ms"] / res["mixed_ms"]
    res["points_per_s_mixed"] = x.shape[0] / (res["mixed_ms"] / 1e3)
    samples["c2w"] = smp
    return res


def _c5(fk, torch, dev, timed, samples, search=True):
    """d=4 Gaussian copula (equicorrelation 0.3, exponential(1) marginals
    centred), N=4e6: one leave-one-out likelihood-and-gradient evaluation on
    each path, and the 20-step bandwidth search (ascent on log h from h=0.5,
    rate 0.5) on the mixed path, timed on the host around the whole search."""
    from paper_2005_03246_gb300 import datagen
    xn = datagen.copula_exp4()["x"]
    x = torch.as_tensor(xn, device=dev)
    n = xn.shape[0]
    h0 = np.full(4, 0.5)
    res = {"workload": "d=4 copula N=4e6, exponential marginals, FP32; LOO likelihood + dL/dh, 16 orthants"}
    for path in ("mixed", "fp64"):
        res["loo_step_%s_ms" % path] = timed(lambda: fk.loo_laplace(x, h0, path=path), reps=1)
    res["loo_mixed_speedup"] = res["loo_step_fp64_ms"] / res["loo_step_mixed_ms"]
    hfin = h0
    if search:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = fk.select_bandwidth_loo(x, h0=0.5, steps=20, lr=0.5, path="mixed")
        torch.cuda.synchronize()
        res["search20_mixed_s"] = time.perf_counter() - t0
        res["search20_fp64_s_estimate"] = 20 * res["loo_step_fp64_ms"] / 1e3
        res["h_final"] = float(hist[-1][0][0])
        res["L_first_last"] = [hist[0][1], hist[-1][1]]
        hfin = hist[-1][0]
    idx = datagen.sample_targets(n, 48, seed=51)
    it = torch.as_tensor(idx, device=dev)
    smp = {"x": xn, "idx": idx, "h": np.asarray(hfin, dtype=np.float64)}
    for path in ("mixed", "fp64"):
        f = fk.kde_laplace(x, hfin, loo=True, path=path)
        smp[path] = f[it].cpu().numpy()
        del f
    samples["c5"] = smp
    return res


def _other_estimators(fk, torch, x, timed):
    """The other estimators on the same d=3, N=1e6 points at the sample points
    (ms, median of the timed runs, L2 flushed): uniform kernel (exact box
    counts; weighted FP64), additive Matern-3/2, full bandwidth matrix,
    Nadaraya-Watson and locally linear regression."""
    y = torch.sin(x.double().sum(dim=1)).to(x.dtype)
    H = np.array([[0.010, 0.004, 0.0], [0.004, 0.012, 0.002], [0.0, 0.002, 0.015]])

    def timed_warm(fn, reps):
        fn()
        torch.cuda.synchronize()
        return timed(fn, reps=reps)

    return {
        "hmatrix": H.tolist(),
        "kde_uniform_counts_ms": timed_warm(lambda: fk.kde_uniform(x, 0.1), reps=3),
        "kde_uniform_weighted_fp64_ms": timed_warm(lambda: fk.kde_uniform(x, 0.1, w=y, path="fp64"), reps=2),
        "kde_matern32_mixed_ms": timed_warm(lambda: fk.kde_matern32(x, 0.1, path="mixed"), reps=3),
        "kde_matern32_fp64_ms": timed_warm(lambda: fk.kde_matern32(x, 0.1, path="fp64"), reps=2),
        "kde_laplace_hmatrix_mixed_ms": timed_warm(lambda: fk.kde_laplace_hmatrix(x, H, path="mixed"), reps=3),
        "kreg_nw_mixed_ms": timed_warm(lambda: fk.kreg_laplace(x, y, 0.1, path="mixed"), reps=3),
        "kreg_loclin_fp64_ms": timed_warm(lambda: fk.kreg_loclin(x, y, 0.1), reps=1),
    }


def _grid_kde_study(fk, torch, x, timed):
    """The grid KDE (exact at the grid points) on grids over the data range,
    interpolated to the N sample points, against the exact sample-point KDE:
    time of the grid KDE and of the interpolation, and the interpolation
    error (relative, on values >= 1e-6 max)."""
    exact = fk.kde_laplace(x, H, path="fp64")
    big = exact >= 1e-6 * exact.max()
    lo = x.min(dim=0).values.double().cpu().numpy()
    hi = x.max(dim=0).values.double().cpu().numpy()
    out = {}
    for m in (64, 128, 256):
        axes = [np.linspace(lo[k], hi[k], m) for k in range(D)]
        t_grid = timed(lambda: fk.kde_grid(x, H, axes, path="mixed"), reps=3)
        f = fk.kde_grid(x, H, axes, path="mixed")
        t_int = timed(lambda: fk.grid_interp(f, axes, x), reps=3)
        fi = fk.grid_interp(f, axes, x)
        rel = ((fi - exact).abs() / exact)[big]
        out["grid%d" % m] = {"kde_grid_ms": t_grid, "interp_ms": t_int,
                             "interp_max_rel_err": float(rel.max()), "interp_median_rel_err": float(rel.median())}
    return out


def _traffic(kernel, alg_bytes):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current sources of that kernel family; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        from paper_2005_03246_gb300 import build as _b
        k = t.get("kernels", {}).get(kernel)
        if not k or k.get("digest") != _b.kernel_digest(kernel):
            return None
        return k["dram_bytes_per_launch"]
    except Exception:
        return None


def _e2e(lib, x_np, grid, args, dev):
    """Same step through the C ABI, inputs and outputs in pinned host memory.
    The three calls are independent, so each runs on its own stream: with
    page-locked host buffers the calls are asynchronous and one call's copies
    overlap the others' kernels.  The timed region ends when all three streams
    have finished (every host output written)."""
    import torch
    from paper_2005_03246_gb300 import _lib
    n = x_np.shape[0]
    xh = torch.empty(x_np.shape, dtype=torch.float32).pin_memory()
    xh.numpy()[:] = x_np
    M = np.array([len(a) for a in grid], dtype=np.int64)
    zh = torch.as_tensor(np.concatenate(grid).astype(np.float64)).pin_memory()
    gpts = int(np.prod(M))
    og = torch.empty((8, gpts), dtype=torch.int64).pin_memory()
    op = torch.empty((8, n), dtype=torch.int64).pin_memory()
    of = torch.empty((n,), dtype=torch.float64).pin_memory()
    h = np.array([H] * D, dtype=np.float64)
    P = ctypes.c_void_p
    streams = [torch.cuda.Stream(dev) for _ in range(3)]
    sp = [P(s.cuda_stream) for s in streams]

    def call():
        # the sample-point counts read tie statistics back once (a host wait), so
        # they are issued last, after the other two calls are enqueued
        rc = lib.fk_kde_laplace(P(xh.data_ptr()), _lib.FK_F32, n, D, None, None, 0, h.ctypes.data_as(P), 0,
                                P(of.data_ptr()), None, 0, None, 0, sp[2])
        _lib.check(rc, "fk_kde_laplace(host)")
        rc = lib.fk_ecdf_grid(P(xh.data_ptr()), _lib.FK_F32, n, D, None, P(zh.data_ptr()),
                              M.ctypes.data_as(P), None, P(og.data_ptr()), 0, None, 0, sp[0])
        _lib.check(rc, "fk_ecdf_grid(host)")
        rc = lib.fk_ecdf_points(P(xh.data_ptr()), _lib.FK_F32, n, D, None, None, 0, None, P(op.data_ptr()), 0,
                                None, 0, sp[1])
        _lib.check(rc, "fk_ecdf_points(host)")
        for s in streams:
            s.synchronize()

    call()
    torch.cuda.synchronize()
    reps = max(2, min(args.steps, 5))
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        call()
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    h2d = 3 * x_np.nbytes + zh.numel() * 8
    d2h = og.numel() * 8 + op.numel() * 8 + of.numel() * 8
    return {"value": n / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": t * 1e3, "streams": 3}


def _scaling_rows(fk, torch, dev, plan, timed, grid=True, reps=3):
    """Runtime versus N on correlated Gaussian data (S_ij = 0.5, FP32): all 2^d
    orthant counts at the sample points, the mixed-path KDE at h = 0.1 and, if
    asked, the grid counts on a grid of ~N points; each time divided by
    N log2^(d-1) N (the divide-and-conquer cost of Sec. 2.2) and, for the grid,
    by N.  plan: [(d, [N, ...]), ...]."""
    rows = []
    r = np.random.default_rng(9)
    for d, sizes in plan:
        S = np.full((d, d), 0.5) + 0.5 * np.eye(d)
        L = np.linalg.cholesky(S)
        for n in sizes:
            xn = (r.standard_normal((n, d)) @ L.T).astype(np.float32)
            x = torch.as_tensor(xn, device=dev)
            shape = n * math.log2(n) ** (d - 1)
            fk.ecdf_points(x)                     # first calls of a shape: set-up outside the timing
            fk.kde_laplace(x, 0.1, path="mixed")
            torch.cuda.synchronize()
            t_pts = timed(lambda: fk.ecdf_points(x), reps)
            t_kde = timed(lambda: fk.kde_laplace(x, 0.1, path="mixed"), reps)
            row = {"d": d, "n": n, "points_ms": t_pts, "kde_mixed_ms": t_kde,
                   "points_ns_per_NlogN": t_pts * 1e6 / shape, "kde_ns_per_NlogN": t_kde * 1e6 / shape}
            if grid:
                m = max(2, int(round(n ** (1.0 / d))))
                axes = [np.linspace(float(xn[:, k].min()), float(xn[:, k].max()), m) for k in range(d)]
                t_grid = timed(lambda: fk.ecdf_grid(x, axes), reps)
                row.update({"grid_ms": t_grid, "grid_points": m ** d, "grid_ns_per_N": t_grid * 1e6 / n})
            rows.append(row)
            del x
            torch.cuda.empty_cache()
    return rows


def run_scaling(args):
    """Runtime versus N at d = 2 ... 6 (the paper's runtime-versus-N study,
    Sec. 4, Tables 1-4); median of 3 runs with L2 flushed; CUDA events."""
    import torch
    import paper_2005_03246_gb300 as fk
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        v = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            r = fn()
            b.record(st)
            b.synchronize()
            v.append(a.elapsed_time(b))
            del r
        return statistics.median(v)

    big = (100_000, 300_000, 1_000_000, 3_000_000)
    plan = [(2, big), (3, big), (4, big), (5, SCALING_HIGH_D[5]), (6, SCALING_HIGH_D[6])]
    rows = _scaling_rows(fk, torch, dev, plan, timed)
    print(json.dumps({"scaling": rows, "data": "synthetic correlated Gaussian, FP32",
                      "shape": "N log2^(d-1) N for the sample-point calls, N for the grid"}), flush=True)
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.scaling:
        return run_scaling(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
