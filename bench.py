"""Benchmark of the aggregate risk analysis hot path on GB300.

One step = one pass of the whole single-layer path over the paper-scale
workload (1,000,000 trials x 1000 events, one layer of 16 ELTs): rebuild the
layer's direct-access table, run the analysis stage for every trial, select
PML 1-in-100/250 and TVaR 99% from the YLT and read them back.  The headline
runs in FP32 with a Kahan-compensated trial sum; the FP64 path and the FP32
path with an FP64 trial sum are timed the same way and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

prints one JSON line.  Under torchrun (N > 1) each rank simulates its own
block of 1,000,000 trials (weak scaling); the ranks' YLTs are gathered once
per step for the PML/TVaR of the whole YET.  ``--impl reference`` times the
CPU oracle on a bounded sample of the same workload instead.

At N = 1 the line also carries three bounded sub-records (skip them with
--no-subrecords): ``portfolio`` (64 uneven layers over a ragged 200,000-trial
YET, batched against plain), ``serving`` (2,000 pricing requests at 200 req/s,
continuous batching against one request per launch, p50/p99) and
``precision_stress`` (each precision mode's error against the FP64 oracle on
the 1M-trial, 32-Pareto-ELT workload).  ``--workload portfolio|serving|
precision_stress`` runs one of those studies alone, in full.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "G event-ELT lookups/s"
UNIT = "G lookups/s"
RPS = [100.0, 250.0]
LEVELS = [0.99]
PRECISION_NAMES = {0: "fp64", 1: "fp32_kahan", 2: "fp32_fp64agg"}
DTYPES = {0: "f64", 1: "f32", 2: "f32"}
FALLBACK_HBM_GBS = 6800.0
CSRC = os.path.join(ROOT, "paper_1308_2066_gb300", "csrc")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--trials", type=int, default=1_000_000)
    p.add_argument("--precision", choices=list(PRECISION_NAMES.values()), default="fp32_kahan")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--workload", choices=["paper_scale", "portfolio", "precision_stress",
                                          "serving"], default="paper_scale")
    p.add_argument("--rates", default="50,200,1000")
    p.add_argument("--seconds-per-rate", type=float, default=8.0)
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--no-subrecords", action="store_true",
                   help="skip the portfolio, serving and precision-stress sub-records")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ---------------------------------------------------------------------------
# measured peaks, clocks, ncu traffic
# ---------------------------------------------------------------------------

def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# Source files of each analysis kernel (its DRAM traffic from ncu goes stale
# when one of them changes).
KERNEL_SOURCES = {
    "k_rows": ["simulate.cu", "rows.cuh", "are_internal.cuh"],
    "k_rows_packed": ["simulate.cu", "rows.cuh", "are_internal.cuh"],
    "k_rows64": ["rows64.cu", "rows.cuh", "fixed.cuh", "are_internal.cuh"],
    "k_simulate_staged": ["simulate.cu", "are_internal.cuh"],
    "k_staged": ["staged.cuh", "staged64.cu", "are_internal.cuh"],
    "k_screen64": ["screen64.cu", "staged.cuh", "are_internal.cuh"],
    "k_sim_items": ["sim_items.cu", "rows.cuh", "are_internal.cuh"],
    "k_simulate": ["simulate.cu", "are_internal.cuh"],
    "k_folded": ["folded.cu", "fixed.cuh", "are_internal.cuh"],
}


def sources_sha(kernel_key: str):
    """Hash of the source files of the kernel named by `kernel_key`."""
    name = kernel_key.split("<")[0]
    files = KERNEL_SOURCES.get(name)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per full launch from the committed ncu summary, if it was
    taken on the kernel's current sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_sha") != sources_sha(kernel_key):
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "25", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(power))}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def algorithmic_bytes(n_events: int, n_trials: int, J: int, elem: int) -> int:
    """YET id (4 B) plus the event's table row in whole 32-byte sectors, per
    event, plus the 8-byte trial loss written per trial."""
    row = math.ceil(J * elem / 32) * 32
    return n_events * (4 + row) + 8 * n_trials


def items_bytes(wl) -> int:
    """Algorithmic bytes of one pass over every layer of a workload."""
    y = wl.yet
    return sum(algorithmic_bytes(y.n_events, y.n_trials, len(L.elts), 4) for L in wl.layers)


def kernel_key(prec: int, J: int, tuned=None, rows=None, ragged=False) -> str:
    """Name of the kernel that runs the analysis stage for this precision
    under the tuned choice (untuned: the register-rows kernels with their
    default batch: one group of 32 events over 32-byte FP32 rows, two
    otherwise).  rows: (row_bytes, packed) from are_layer_rows, which names
    the packed-row instances; ragged: the YET has trials of varying length."""
    if prec == "folded":
        return "k_folded<fixed,smem_bits>"
    t = tuned or {}
    rb, packed = rows if rows else (None, False)
    u = t.get("rows_in_flight") or (1 if prec != 0 and (rb == 32 or (rb is None and J <= 8)) else 2)
    cur = "ragged" if ragged else "fixed"
    if prec == 0:
        jp = math.ceil(J / 4) * 4
        kind = t.get("kernel", 2)
        if kind == 3:
            return f"k_screen64<{8 if J <= 8 else 16 if J <= 16 else 32},{cur}>"
        if kind == 1:
            return f"k_staged<double,{jp},{cur},ylt>"
        return f"k_rows64<{(rb or 64) // 8},{u},{cur}>"
    jp = 8 if J <= 8 else 16 if J <= 16 else 32
    kind = t.get("kernel", 2)
    if kind == 0:
        return f"k_sim_items<{jp},{u},{prec},{cur}>"
    if kind == 2:
        if packed:
            return f"k_rows_packed<{rb // 4},{u},{prec},{cur}>"
        return f"k_rows<{jp},{u},{prec},{cur}>"
    return f"k_simulate_staged<{jp},{prec},{cur},epl{2 if u == 2 else 1}>"


def layer_rows(are, ctx, layer, yet, prec, tuned=None):
    """(row_bytes, packed) of the rows the analysis of this layer reads per
    occurrence under the tuned kernel choice (the library's answer)."""
    return are.are_layer_rows(ctx, layer, yet, prec, (tuned or {}).get("kernel", -1))


class Resident:
    """The workload loaded once into a context (device-resident inputs)."""

    def __init__(self, are, ctx, wl, torch):
        y = wl.yet
        self.wl, self.are, self.ctx = wl, are, ctx
        ids = torch.from_numpy(y.ids).cuda()
        self.yet = are.are_load_yet(ctx, y.catalog, y.n_trials, None, y.k, ids)
        del ids
        self.elts = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share)
                     for e in wl.elts]
        L = wl.layers[0]
        self.layer = are.are_define_layer(ctx, self.elts, L.occ_r, L.occ_l, L.agg_r, L.agg_l)


class StepMeasures:
    """A step's PML/TVaR: selected into device arrays (the call only
    enqueues) and copied to pinned host memory on the step's stream, so
    consecutive steps queue back to back; read after the stream is done."""

    def __init__(self, torch):
        self.d_pml = torch.empty(len(RPS), dtype=torch.float64, device="cuda")
        self.d_tv = torch.empty(len(LEVELS), dtype=torch.float64, device="cuda")
        self.h_pml = torch.empty(len(RPS), dtype=torch.float64, pin_memory=True)
        self.h_tv = torch.empty(len(LEVELS), dtype=torch.float64, pin_memory=True)

    def select(self, are, torch, ctx, ylt, n, stream):
        are.are_risk_measures(ctx, ylt, n, RPS, LEVELS, stream, out=(self.d_pml, self.d_tv))
        with torch.cuda.stream(stream):
            self.h_pml.copy_(self.d_pml, non_blocking=True)
            self.h_tv.copy_(self.d_tv, non_blocking=True)

    def values(self):
        return [float(x) for x in self.h_pml], [float(x) for x in self.h_tv]


def time_path(are, torch, res, prec, steps, warmup, stream, ylt, gather=None, world=1):
    """Run warmup + timed steps of one precision; returns timing dict."""
    ctx, wl = res.ctx, res.wl
    n = wl.yet.n_trials
    sim_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
    meas = StepMeasures(torch)

    def step(i=None):
        are.are_prepare(ctx, res.layer, res.yet, prec, stream)
        if i is not None:
            sim_ev[i][0].record(stream)
        are.are_simulate(ctx, res.layer, res.yet, 0, n, prec, ylt, stream)
        if i is not None:
            sim_ev[i][1].record(stream)
        if gather is not None:
            with torch.cuda.stream(stream):
                full = gather(ylt)
            meas.select(are, torch, ctx, full, full.numel(), stream)
        else:
            meas.select(are, torch, ctx, ylt, n, stream)

    for _ in range(warmup):
        step()
    barrier(world)
    torch.cuda.synchronize()
    l0 = are.are_launch_count(ctx)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        start.record(stream)
        for i in range(steps):
            step(i)
        end.record(stream)
        end.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    launches = are.are_launch_count(ctx) - l0
    ms = start.elapsed_time(end)
    sim_ms = float(np.mean([a.elapsed_time(b) for a, b in sim_ev]))
    pml, tvar = meas.values()
    return {"ms": ms, "sim_ms": sim_ms, "launches": launches, "clocks": clk.summary(),
            "pml": pml, "tvar": tvar}


def time_folded(are, torch, res, steps, warmup, stream, ylt, gather=None, world=1):
    """The folded-table variant: rebuild the folded table, one trial pass,
    PML/TVaR, per step."""
    ctx, wl = res.ctx, res.wl
    n = wl.yet.n_trials
    sim_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
    meas = StepMeasures(torch)

    def step(i=None):
        are.are_prepare_folded(ctx, res.layer, res.yet, stream)
        if i is not None:
            sim_ev[i][0].record(stream)
        are.are_simulate_folded(ctx, res.layer, res.yet, 0, n, ylt, stream)
        if i is not None:
            sim_ev[i][1].record(stream)
        if gather is not None:
            with torch.cuda.stream(stream):
                full = gather(ylt)
            meas.select(are, torch, ctx, full, full.numel(), stream)
        else:
            meas.select(are, torch, ctx, ylt, n, stream)

    for _ in range(warmup):
        step()
    barrier(world)
    torch.cuda.synchronize()
    l0 = are.are_launch_count(ctx)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        start.record(stream)
        for i in range(steps):
            step(i)
        end.record(stream)
        end.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    return {"ms": start.elapsed_time(end),
            "sim_ms": float(np.mean([a.elapsed_time(b) for a, b in sim_ev])),
            "launches": are.are_launch_count(ctx) - l0, "clocks": clk.summary(),
            "pml": meas.values()[0], "tvar": meas.values()[1]}


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, torch) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


SHAPE_NAMES = {0: "16-byte loads, lane reads its row's id",
               1: "32-byte loads, ids shuffled from one coalesced read per 32 events",
               2: "cp.async rows staged in shared memory"}


def roofline(n_events, n_trials, J, prec, sim_ms, tuned=None, ceiling=None, rows=None):
    """Roofline of the analysis kernel.  Its table rows are gathered from the
    L2-resident table, so the bound that applies is the gather ceiling: the
    same id stream and row reads with no arithmetic, measured live in this
    run over every launch shape of are_gather_ceiling for the kernel's row
    size.  achieved and peak are the algorithmic bytes (4 B id + the row the
    kernel reads per event, 8 B per trial) over the kernel's time and over
    the ceiling's time, so frac = the kernel's rows/s over the ceiling's.
    hbm_formula_frac puts the dense-row formula's bytes (the row of J entries of
    the precision, in whole 32-B sectors) over the measured HBM copy
    bandwidth (above 1: the rows are not HBM traffic); dram_frac is the
    ncu-measured DRAM traffic of one launch over the kernel's time, over
    that bandwidth."""
    hbm, src = hbm_peak()
    rb = rows[0]
    bytes_ = n_events * (4 + rb) + 8 * n_trials
    dense_bytes = algorithmic_bytes(n_events, n_trials, J, 8 if prec == 0 else 4)
    secs = sim_ms * 1e-3
    achieved = bytes_ / secs / 1e9
    key = kernel_key(prec, J, tuned, rows)
    traffic = ncu_traffic(key)
    best, shapes = ceiling
    rate = n_events / secs
    top = max(shapes, key=lambda x: x[3])
    return {"bound": "l2_gather", "achieved": round(achieved, 1),
            "peak": round(bytes_ / (n_events / best) / 1e9, 1), "unit": "GB/s",
            "frac": round(rate / best, 4), "traffic": traffic, "kernel": key,
            "algorithmic_bytes_per_launch": bytes_,
            "dense_formula_bytes_per_launch": dense_bytes,
            "peak_source": ("measured live in this run: best of %d launch shapes of the gather "
                            "ceiling (ids + table rows, no arithmetic) on this YET" % len(shapes)),
            "hbm_formula_frac": round(dense_bytes / secs / 1e9 / hbm, 4),
            "dram_frac": (round(traffic / secs / 1e9 / hbm, 4) if traffic else None),
            "hbm_peak": hbm, "hbm_peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json)",
            "l2_gather": {"row_bytes": rb, "packed_rows": rows[1],
                          "achieved_rows_per_s": round(rate, 1),
                          "ceiling_rows_per_s": round(best, 1),
                          "ceiling_shape": {"kind": SHAPE_NAMES[top[0]], "in_flight": top[1],
                                            "blocks_per_sm": top[2]},
                          "shapes_timed": len(shapes)}}


def folded_roofline(n_events, n_trials, sim_ms):
    """The folded table's trial pass: HBM traffic is the id stream and the
    YLT; the values of the few events with h > 0 come from L2."""
    peak, src = hbm_peak()
    bytes_ = 4 * n_events + 8 * n_trials
    achieved = bytes_ / (sim_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": ncu_traffic(kernel_key("folded", 0)),
            "kernel": kernel_key("folded", 0), "algorithmic_bytes_per_launch": bytes_,
            "peak_source": f"{src} HBM copy bandwidth",
            "note": "algorithmic bytes = 4 B id per event + 8 B per trial"}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline, and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(wl, seconds: float, probe_trials: int = 200):
    """Time the oracle on a prefix of the workload's trials sized to take about
    `seconds`; returns (lookups/s, trials timed, threads, wall seconds)."""
    import oracle
    oracle.build()
    J = len(wl.layers[0].elts)
    k = wl.yet.k
    t0 = time.perf_counter()
    oracle.simulate_layer(wl, trials=np.arange(probe_trials))
    per_trial = (time.perf_counter() - t0) / probe_trials
    n = int(min(wl.yet.n_trials, max(probe_trials, seconds / max(per_trial, 1e-9))))
    t0 = time.perf_counter()
    oracle.simulate_layer(wl, trials=np.arange(n))
    dt = time.perf_counter() - t0
    return n * k * J / dt, n, oracle.max_threads(), dt


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    budget_s = 150.0
    per_step_s = min(2.0, budget_s / max(1, args.steps + args.warmup))
    probe = W.paper_scale(n_trials=200)
    t0 = time.perf_counter()
    oracle.simulate_layer(probe)
    per_trial = (time.perf_counter() - t0) / 200
    n = int(max(50, min(args.trials, per_step_s / max(per_trial, 1e-9))))
    wl = W.paper_scale(n_trials=n)
    J, k = len(wl.layers[0].elts), wl.yet.k
    for _ in range(args.warmup):
        oracle.simulate_layer(wl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.simulate_layer(wl)
        oracle.risk_measures(r.ylt, RPS, LEVELS)
    dt = time.perf_counter() - t0
    value = args.steps * n * k * J / dt / 1e9
    sample = (f"first {n} trials of the 1,000,000 x 1000-event, 16-ELT workload per step "
              f"(full sort for PML/TVaR of that sample)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper_scale_1000000_x_1000_j16", "sample_trials": n,
                       "precision": "fp64 oracle"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# end-to-end through the C ABI with host buffers
# ---------------------------------------------------------------------------

def run_e2e(are, torch, ctx, wl, prec, steps, warmup, world):
    """Per step, from pinned host memory through the public API: load the
    ELTs, define the layer, build its table, analyse the host-resident YET
    (its copy to the device overlapped with the analysis, chunk by chunk),
    select PML/TVaR and read them back.  The YET is held in host memory with
    its ids packed in the bits the catalog needs (are_pack_ids, once, before
    the timed steps); the same steps over int32 ids are reported beside."""
    y = wl.yet
    L = wl.layers[0]
    bits = max(1, int(y.catalog - 1).bit_length())
    words = are.packed_words(y.n_events, bits)
    packed = torch.empty(words, dtype=torch.int32, pin_memory=True)
    are.are_pack_ids(ctx, y.ids, bits, packed.data_ptr())
    ids_pinned = torch.from_numpy(y.ids).pin_memory()
    elt_bytes = sum(e.ids.nbytes + e.losses.nbytes for e in wl.elts)
    ylt = torch.empty(y.n_trials, dtype=torch.float64, device="cuda")
    d2h = 8 * (len(RPS) + len(LEVELS))

    def timed(analyse):
        def step():
            elts = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share)
                    for e in wl.elts]
            layer = are.are_define_layer(ctx, elts, L.occ_r, L.occ_l, L.agg_r, L.agg_l)
            analyse(layer)
            are.are_risk_measures(ctx, ylt, y.n_trials, RPS, LEVELS)
            are.are_free_layer(ctx, layer)
            for h in elts:
                are.are_free_elt(ctx, h)

        for _ in range(warmup):
            step()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, world, torch)

    dt = timed(lambda layer: are.are_simulate_streamed_packed(
        ctx, layer, y.catalog, y.n_trials, None, y.k, packed.data_ptr(), bits, prec, ylt))
    dt32 = timed(lambda layer: are.are_simulate_streamed(
        ctx, layer, y.catalog, y.n_trials, None, y.k, ids_pinned, prec, ylt))
    J = len(L.elts)
    value = world * steps * y.n_events * J / dt / 1e9
    return {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": int(4 * words + elt_bytes),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(dt / steps * 1e3, 3),
            "how": (f"are_load_elt x J, are_define_layer, are_simulate_streamed_packed (host YET with "
                    f"{bits}-bit ids, copy overlapped with the analysis), are_risk_measures, frees"),
            "int32_ids": {"value": round(world * steps * y.n_events * J / dt32 / 1e9, 3),
                          "ms_per_step": round(dt32 / steps * 1e3, 3),
                          "h2d_bytes_per_step": int(y.ids.nbytes + elt_bytes),
                          "how": "the same steps with are_simulate_streamed over int32 ids"}}


# ---------------------------------------------------------------------------
# the per-occurrence outputs and the compact table on the paper-scale layer
# ---------------------------------------------------------------------------

def next_record(are, torch, res, steps, warmup):
    """Per-occurrence outputs (the marginal of every occurrence, each trial's
    largest occurrence loss and the YLT) in FP64 and FP32 + Kahan, and the
    FP32 + Kahan analysis over the compact table (a row index and rows only
    for the events some ELT holds), timed with CUDA events on the resident
    paper-scale workload and checked against the direct analysis's YLT."""
    ctx, wl = res.ctx, res.wl
    y = wl.yet
    n, J = y.n_trials, len(wl.layers[0].elts)
    stream = torch.cuda.Stream()
    hbm, _ = hbm_peak()
    out = {}

    def timed(fn):
        for _ in range(warmup):
            fn()
        evs = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ylt = torch.empty(n, dtype=torch.float64, device="cuda")
    marg = torch.empty(y.n_events, dtype=torch.float64, device="cuda")
    occ_max = torch.empty(n, dtype=torch.float64, device="cuda")
    for p in (0, 1):
        are.are_prepare(ctx, res.layer, res.yet, p, stream)
        are.are_simulate(ctx, res.layer, res.yet, 0, n, p, ref, stream)
        ms = timed(lambda: are.are_simulate_occurrences(ctx, res.layer, res.yet, 0, n, p, marg, occ_max,
                                                       ylt, stream))
        torch.cuda.synchronize()
        diff = float(((ylt - ref).abs() / ref.abs().clamp_min(1e-300)).max())
        hbm_bytes = y.n_events * (4 + 8) + n * 16   # ids in, marginals, maxima and YLT out
        out[f"per_occurrence_outputs_{PRECISION_NAMES[p]}"] = {
            "ms": round(ms, 4), "value": round(y.n_events * J / (ms * 1e-3) / 1e9, 3),
            "unit": UNIT, "hbm_bytes_per_launch": hbm_bytes,
            "hbm_frac": round(hbm_bytes / (ms * 1e-3) / 1e9 / hbm, 4),
            "ylt_rel_diff_max_vs_analysis": diff,
            "what": "are_simulate_occurrences: every occurrence's marginal (8 B), each trial's "
                    "largest occurrence loss and the YLT"}
    del marg
    torch.cuda.empty_cache()
    are.are_prepare(ctx, res.layer, res.yet, 1, stream)
    are.are_simulate(ctx, res.layer, res.yet, 0, n, 1, ref, stream)
    are.are_set_table_layout(ctx, res.layer, are.ARE_LAYOUT_COMPACT)
    try:
        are.are_prepare(ctx, res.layer, res.yet, 1, stream)
        ms = timed(lambda: are.are_simulate(ctx, res.layer, res.yet, 0, n, 1, ylt, stream))
        torch.cuda.synchronize()
        diff = float(((ylt - ref).abs() / ref.abs().clamp_min(1e-300)).max())
        out["compact_table_fp32_kahan"] = {
            "ms": round(ms, 4), "value": round(y.n_events * J / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "ylt_rel_diff_max_vs_direct": diff,
            "what": "the compact layout (a row index over the catalog and rows of the events some "
                    "ELT holds) on the staged kernel: the rows of absent events are not read"}
    finally:
        are.are_set_table_layout(ctx, res.layer, are.ARE_LAYOUT_DIRECT)
    return out


# ---------------------------------------------------------------------------
# portfolio batching: 64 uneven layers over one ragged YET
# ---------------------------------------------------------------------------

def portfolio_kernel_name(tuned, prec) -> str:
    """What runs the batched analysis under the tuned choice."""
    kind = (tuned or {}).get("kernel", 2)
    u = (tuned or {}).get("rows_in_flight") or "U"   # untuned: 1 over 32-byte rows, else 2
    if kind == 0:
        return (f"k_sim_items<jp,{u},{prec},ragged>: one persistent launch per table width, "
                f"{(tuned or {}).get('trials_per_item')} trials per work item")
    if kind == 2:
        return (f"k_rows<jp,{u},{prec},ragged> (k_rows_packed<pw,{u},{prec},ragged> over the packed rows "
                f"of the layers of more than 8 ELTs): one launch per layer, back to back in the graph")
    return f"k_simulate_staged<jp,{prec},ragged,epl{u}>: one launch per layer, back to back in the graph"


def portfolio_record(are, torch, prec, steps, warmup, tune=True, variants=True, rank=0, world=1,
                     local_rank=0, n_trials=200_000):
    """Portfolio of 64 uneven layers (1..32 ELTs from a pool of 256) over a
    ragged 200,000-trial YET: the batched form (every table rebuilt, one
    graph-replayed analysis of all layers, one batched PML/TVaR) against the
    plain form (per layer: repack, are_simulate, are_risk_measures).  Under
    torchrun each rank takes whole layers (no exchange in the step)."""
    wl = W.portfolio(n_trials=min(n_trials, 200_000))
    all_layers = wl.layers
    from paper_1308_2066_gb300.sharding import layer_shard
    mine = layer_shard([len(L.elts) for L in all_layers], world, rank)
    wl.layers = [all_layers[i] for i in mine]
    y = wl.yet
    ctx = are.are_create(local_rank)
    try:
        ids = torch.from_numpy(y.ids).cuda()
        off = torch.from_numpy(y.offsets).cuda()
        yet = are.are_load_yet(ctx, y.catalog, y.n_trials, off, 0, ids)
        del ids, off
        elts = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share) for e in wl.elts]
        layers = [are.are_define_layer(ctx, [elts[m] for m in L.elts], L.occ_r, L.occ_l, L.agg_r,
                                       L.agg_l) for L in wl.layers]
        n = y.n_trials
        stream = torch.cuda.Stream()
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in layers]
        tuned = are.are_autotune(ctx, layers, yet, prec, stream) if tune else None
        lookups = sum(y.n_events * len(L.elts) for L in all_layers)   # the whole portfolio

        def batched():
            for h in layers:
                are.are_prepare(ctx, h, yet, prec, stream)
            are.are_simulate_portfolio(ctx, layers, yet, 0, n, prec, outs, stream)
            return are.are_risk_measures_batch(ctx, outs, n, RPS, LEVELS, stream)

        def plain():
            for h, o in zip(layers, outs):
                are.are_prepare(ctx, h, yet, prec, stream)
                are.are_simulate(ctx, h, yet, 0, n, prec, o, stream)
                are.are_risk_measures(ctx, o, n, RPS, LEVELS, stream)

        def timed(fn, k):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            barrier(world)
            l0 = are.are_launch_count(ctx)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(local_rank) as clk:
                a.record(stream)
                for _ in range(k):
                    fn()
                b.record(stream)
                b.synchronize()
            barrier(world)
            ms = max_over_ranks(a.elapsed_time(b) / k, world, torch)
            return ms, are.are_launch_count(ctx) - l0, clk.summary()

        # the analysis alone (one graph replay of every layer), for the roofline
        sim = []
        for _ in range(warmup + steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            are.are_simulate_portfolio(ctx, layers, yet, 0, n, prec, outs, stream)
            e1.record(stream)
            sim.append((e0, e1))
        torch.cuda.synchronize()
        sim_ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in sim[warmup:]])),
                                world, torch)
        ms_b, launches, clocks = timed(batched, steps)
        ms_p, launches_p, _ = timed(plain, max(1, steps // 2))
        folded = None
        if variants:
            def folded_fn():   # each layer's folded table, one exact pass per layer
                for h, o in zip(layers, outs):
                    are.are_prepare_folded(ctx, h, yet, stream)
                    are.are_simulate_folded(ctx, h, yet, 0, n, o, stream)
                return are.are_risk_measures_batch(ctx, outs, n, RPS, LEVELS, stream)
            ms_f, launches_f, _ = timed(folded_fn, max(1, steps // 2))
            folded = {"ms_per_step": round(ms_f, 4),
                      "value": round(lookups / (ms_f * 1e-3) / 1e9, 3),
                      "value_unit": "G event-ELT lookups/s equivalent", "gpu_launches": launches_f,
                      "what": ("per layer: FP64 folded table (one lookup per occurrence) and one "
                               "exact trial pass; batched PML/TVaR")}
        pml, tv = batched()
        per_layer = {i: ([float(x) for x in pml[k]], [float(x) for x in tv[k]])
                     for k, i in enumerate(mine)}
        if world > 1:
            from paper_1308_2066_gb300.sharding import gather_results
            per_layer = dict(enumerate(gather_results(per_layer, len(all_layers))))
        # the gather ceiling of every row size on this YET: the time it would
        # take for every layer's rows, against the analysis' time
        ceil = {}
        t_ceil = 0.0
        for h in layers:
            rb, _ = layer_rows(are, ctx, h, yet, prec, tuned)
            if rb not in ceil:
                ceil[rb] = are.are_gather_ceiling(ctx, yet, rb, 0, n, reps=2)
            t_ceil += y.n_events / ceil[rb]
        hbm, src = hbm_peak()
        mine_bytes = sum(algorithmic_bytes(y.n_events, y.n_trials, len(L.elts), 4 if prec else 8)
                         for L in wl.layers)
        roof = {"bound": "l2_gather", "achieved": round(mine_bytes / (sim_ms * 1e-3) / 1e9, 1),
                "peak": round(mine_bytes / t_ceil / 1e9, 1), "unit": "GB/s",
                "frac": round(t_ceil / (sim_ms * 1e-3), 4), "traffic": None,
                "kernel": portfolio_kernel_name(tuned, prec),
                "algorithmic_bytes_per_launch": mine_bytes, "sim_ms": round(sim_ms, 4),
                "peak_source": "measured live: the gather ceiling of each layer's row size on this YET",
                "hbm_formula_frac": round(mine_bytes / (sim_ms * 1e-3) / 1e9 / hbm, 4)}
        return {
            "metric": METRIC, "value": round(lookups / (ms_b * 1e-3) / 1e9, 3), "unit": UNIT,
            "n_gpus": world, "steps": steps, "warmup": warmup, "ms_per_step": round(ms_b, 4),
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": DTYPES[prec],
            "data": "synthetic: seeded ragged Poisson(1000) YET, lognormal ELT pool",
            "config": {"workload": wl.name, "trials": n, "events": y.n_events,
                       "layers": len(all_layers), "elts_per_layer": [len(L.elts) for L in all_layers],
                       "precision": PRECISION_NAMES[prec],
                       "step": "repack every table + one graph-replayed analysis of every layer + "
                               "batched PML/TVaR",
                       "l2": "inputs larger than L2 (0.8 GB YET streamed once per layer)",
                       "parallelism": f"whole layers per GPU x{world} (greedy by ELT count)"},
            "roofline": roof,
            "plain": {"ms_per_step": round(ms_p, 4), "value": round(lookups / (ms_p * 1e-3) / 1e9, 3),
                      "gpu_launches": launches_p,
                      "how": "64 x (repack + are_simulate + are_risk_measures)"},
            "speedup_vs_plain": round(ms_p / ms_b, 3),
            "folded_variant": folded, "tuned": tuned, "kernel": portfolio_kernel_name(tuned, prec),
            "gpu_launches": launches, "clocks": clocks,
            "pml_layer0": per_layer[0][0], "tvar_layer0": per_layer[0][1]}
    finally:
        are.are_destroy(ctx)


def run_portfolio(args):
    import torch
    import paper_1308_2066_gb300 as are
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    prec = {v: k for k, v in PRECISION_NAMES.items()}[args.precision]
    line = portfolio_record(are, torch, prec, args.steps, args.warmup, tune=not args.no_tune,
                            variants=not args.no_variants, rank=rank, world=world,
                            local_rank=local_rank, n_trials=args.trials)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# precision modes: 32 Pareto ELTs, long ragged trials, errors vs the oracle
# ---------------------------------------------------------------------------

def precision_record(are, torch, steps, warmup, tune=True, compact=True, n_trials=1_000_000,
                     n_sample=2000):
    """Each precision mode on the precision-stress workload (1M ragged trials
    of Poisson(1000) <= 3000 events over a 2M-event catalog, 32 Pareto(1.3)
    ELTs, neutral terms: whole-trial sums reach the YLT): analysis time, and
    the error against the FP64 oracle of the YLT on sampled trials and of
    PML/TVaR through the tail trials."""
    import oracle
    wl = W.precision_stress(n_trials=min(n_trials, 1_000_000))
    y = wl.yet
    ctx = are.are_create(0)
    try:
        ids = torch.from_numpy(y.ids).cuda()
        off = torch.from_numpy(y.offsets).cuda()
        yet = are.are_load_yet(ctx, y.catalog, y.n_trials, off, 0, ids)
        del ids, off
        elts = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share) for e in wl.elts]
        L = wl.layers[0]
        layer = are.are_define_layer(ctx, elts, L.occ_r, L.occ_l, L.agg_r, L.agg_l)
        n = y.n_trials
        stream = torch.cuda.Stream()
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        sample = np.sort(np.random.default_rng(7).choice(n, min(n, n_sample), replace=False))
        ref = oracle.simulate_layer(wl, trials=sample)
        rows = {}
        kahan_ylt = None

        def timed(p):
            evs = []
            for _ in range(warmup + steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                are.are_simulate(ctx, layer, yet, 0, n, p, out, stream)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            return float(np.mean([a.elapsed_time(b) for a, b in evs[warmup:]]))

        for p in (0, 2, 1):
            tuned = are.are_autotune(ctx, [layer], yet, p, stream) if tune else None
            ms = timed(p)
            got = out.cpu().numpy()
            if p == 1:
                kahan_ylt = got.copy()
            d = np.abs(got[sample] - ref.ylt)
            rel = d / np.maximum(np.abs(ref.ylt), 1e-300)
            pml, tv = are.are_risk_measures(ctx, out, n, RPS, LEVELS, stream)
            # PML/TVaR of the oracle over the GPU's tail trials (the top 1.25 m)
            m_max = oracle.rank_for_level(n, LEVELS[0])
            cand = np.sort(np.argsort(-got)[: m_max + m_max // 4])
            rc = oracle.simulate_layer(wl, trials=cand)
            full = np.zeros(n)
            full[cand] = rc.ylt
            rp, rt = oracle.risk_measures(full, RPS, LEVELS)
            rows[PRECISION_NAMES[p]] = {
                "sim_ms": round(ms, 4), "tuned": tuned,
                "kernel": kernel_key(p, len(L.elts), tuned, layer_rows(are, ctx, layer, yet, p, tuned),
                                     ragged=True),
                "value": round(y.n_events * len(L.elts) / (ms * 1e-3) / 1e9, 3),
                "ylt_rel_err_max": float(rel.max()), "ylt_rel_err_median": float(np.median(rel)),
                "pml": [float(x) for x in pml], "pml_oracle": [float(x) for x in rp],
                "pml_rel_err": [float(abs(a - b) / b) for a, b in zip(pml, rp)],
                "tvar": [float(x) for x in tv], "tvar_oracle": [float(x) for x in rt],
                "tvar_rel_err": [float(abs(a - b) / b) for a, b in zip(tv, rt)]}
        if compact:
            # the compact table (row index + rows of the events in some ELT): a
            # variant that does not read the rows of events absent from every ELT
            are.are_set_table_layout(ctx, layer, are.ARE_LAYOUT_COMPACT)
            are.are_prepare(ctx, layer, yet, 1, stream)
            ms_c = timed(1)
            got = out.cpu().numpy()
            rows["fp32_kahan_compact_variant"] = {
                "sim_ms": round(ms_c, 4),
                "value": round(y.n_events * len(L.elts) / (ms_c * 1e-3) / 1e9, 3),
                "ylt_rel_err_max_vs_direct": float(np.max(np.abs(got - kahan_ylt) /
                                                          np.maximum(np.abs(kahan_ylt), 1e-300))),
                "what": "compact table on the staged kernel: row index over the 2M catalog + rows "
                        "of the events present in some ELT; rows of absent events are not read"}
            are.are_set_table_layout(ctx, layer, are.ARE_LAYOUT_DIRECT)
        return {"workload": wl.name, "trials": n, "events": y.n_events, "elts": len(L.elts),
                "sample_trials": int(sample.size),
                "errors_against": "FP64 oracle: sampled trials one by one; PML/TVaR over the "
                                  "oracle's losses of the GPU's top 1.25 m trials",
                "precisions": rows}
    finally:
        are.are_destroy(ctx)


def run_precision_stress(args):
    import torch
    import paper_1308_2066_gb300 as are
    torch.cuda.set_device(0)
    rec = precision_record(are, torch, args.steps, args.warmup, tune=not args.no_tune,
                           n_trials=args.trials)
    head = rec["precisions"][args.precision]
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["sim_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[{v: k for k, v in PRECISION_NAMES.items()}[args.precision]],
            "data": "synthetic: ragged Poisson(1000)<=3000 YET over 2M events, 32 Pareto(1.3) ELTs",
            "config": {"workload": rec["workload"], "trials": rec["trials"], "events": rec["events"],
                       "elts": rec["elts"], "sample_trials": rec["sample_trials"]},
            "precisions": rec["precisions"]}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: Poisson stream of pricing requests over a resident YET and ELT pool
# ---------------------------------------------------------------------------

def serve_stream(are, ctx, hs, reqs, one_at_a_time, prec, k, folded=False, least_work_first=False):
    """Submit each request at its arrival time, collect every result; returns
    per-request latencies (ms) and the wall time from first submit to last result."""
    import queue
    tickets = queue.Queue()
    out = []
    are.are_server_start(ctx, hs["yet"], max_inflight=32, max_pending=100000,
                         arena_bytes=6 << 30, one_at_a_time=one_at_a_time, precision=prec,
                         folded=folded, least_work_first=least_work_first)

    def collect():
        while True:
            item = tickets.get()
            if item is None:
                return
            r, t = item
            res = are.are_wait(ctx, t, 600_000_000)
            out.append((res["total_us"] / 1e3, res["status"], r, res))

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for r in reqs:
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        L = r.layer
        t = are.are_submit(ctx, [hs["elts"][m] for m in L.elts], L.occ_r, L.occ_l, L.agg_r,
                           L.agg_l, r.n_trials, RPS, LEVELS)
        tickets.put((r, t))
    tickets.put(None)
    th.join()
    wall = time.perf_counter() - t0
    are.are_server_stop(ctx)
    lat = np.array([o[0] for o in out])
    assert all(o[1] == 0 for o in out), "a request failed"
    lookups = sum(r.n_trials * k * len(r.layer.elts) for r in reqs)
    return {"requests": len(reqs), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3),
            "throughput_req_s": round(len(reqs) / wall, 2),
            "g_lookups_s": round(lookups / wall / 1e9, 2)}, out


def serving_record(are, torch, prec, rates, seconds_per_rate, min_requests=200,
                   max_requests=2000, folded=True, n_trials=1_000_000):
    """Poisson streams of pricing requests (1..16 random ELTs of a pool of
    256, fresh layer terms, 1e4..1e6 trials) over a resident 1M x 1000 YET:
    p50/p99 latency and throughput with continuous batching against one
    request per launch, on the same request stream."""
    wl = W.serving_pool(n_trials=min(n_trials, 1_000_000))
    y = wl.yet
    ctx = are.are_create(0)
    try:
        ids = torch.from_numpy(y.ids).cuda()
        hs = {"yet": are.are_load_yet(ctx, y.catalog, y.n_trials, None, y.k, ids)}
        del ids
        hs["elts"] = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share)
                      for e in wl.elts]
        pooled = np.concatenate([e.losses for e in wl.elts[:16]])
        rows = {}
        for i, rate in enumerate(rates):
            n_req = int(min(max_requests, max(min_requests, rate * seconds_per_rate)))
            reqs = W.pricing_requests(n_req, rate, pool=len(wl.elts), max_trials=y.n_trials,
                                      stream=10 + i, pooled_losses=pooled)
            l0 = are.are_launch_count(ctx)
            batched, _ = serve_stream(are, ctx, hs, reqs, False, prec, y.k)
            batched["gpu_launches"] = are.are_launch_count(ctx) - l0
            single, _ = serve_stream(are, ctx, hs, reqs, True, prec, y.k)
            lwf, _ = serve_stream(are, ctx, hs, reqs, False, prec, y.k, least_work_first=True)
            lwf["what"] = "continuous batching, the budget to the least remaining work first"
            row = {"continuous_batching": batched, "one_request_per_launch": single,
                   "p99_batched_over_single": round(batched["p99_ms"] / single["p99_ms"], 4),
                   "least_work_first": lwf}
            if folded:
                f, _ = serve_stream(are, ctx, hs, reqs, False, prec, y.k, folded=True)
                f["what"] = ("variant: continuous batching on folded tables (FP64 occurrence loss "
                             "per catalog event, exact trial sums, one lookup per occurrence)")
                row["folded_continuous_batching_variant"] = f
            rows[str(int(rate))] = row
        return {"workload": wl.name, "request_trials": "log-uniform 1e4..1e6 (YET prefix)",
                "request_elts": "1..16 of the pool", "measures": "PML 100/250, TVaR 99",
                "precision": PRECISION_NAMES[prec], "rates": rows}
    finally:
        are.are_destroy(ctx)


def run_serving(args):
    import torch
    import paper_1308_2066_gb300 as are
    torch.cuda.set_device(0)
    prec = {v: k for k, v in PRECISION_NAMES.items()}[args.precision]
    rates = [float(x) for x in args.rates.split(",")]
    rec = serving_record(are, torch, prec, rates, args.seconds_per_rate, n_trials=args.trials)
    rows = rec["rates"]
    head = rows.get("200", next(iter(rows.values())))["continuous_batching"]
    line = {"metric": "p99 pricing latency", "value": head["p99_ms"], "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[prec],
            "data": "synthetic: resident 1M x 1000 YET, 256 lognormal ELTs, Poisson arrivals",
            "config": {k: v for k, v in rec.items() if k != "rates"} | {"headline_rate_req_s": 200},
            "rates": rows}
    print(json.dumps(line), flush=True)


def subrecords(are, torch, args):
    """The portfolio, serving and precision-stress studies, each bounded to
    a few tens of seconds, for the default run's line."""
    out = {}
    prec = {v: k for k, v in PRECISION_NAMES.items()}[args.precision]
    for name, fn in (
            ("portfolio", lambda: portfolio_record(are, torch, prec, 5, 2, variants=False)),
            ("serving", lambda: serving_record(are, torch, prec, [50.0, 200.0], 20.0,
                                               min_requests=1000, max_requests=2000,
                                               folded=False)),
            ("precision_stress", lambda: precision_record(are, torch, 5, 2, compact=False))):
        t0 = time.perf_counter()
        try:
            rec = fn()
        except Exception as e:   # the headline line is still printed
            rec = {"error": f"{type(e).__name__}: {e}"}
        rec["wall_s"] = round(time.perf_counter() - t0, 1)
        out[name] = rec
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "portfolio":
        return run_portfolio(args)
    if args.workload == "precision_stress":
        return run_precision_stress(args)
    if args.workload == "serving":
        return run_serving(args)
    import torch
    import paper_1308_2066_gb300 as are

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    prec = {v: k for k, v in PRECISION_NAMES.items()}[args.precision]

    wl = W.paper_scale(n_trials=args.trials, shard=rank)
    y = wl.yet
    J = len(wl.layers[0].elts)
    ctx = are.are_create(local_rank)
    res = Resident(are, ctx, wl, torch)
    stream = torch.cuda.Stream()
    ylt = torch.empty(y.n_trials, dtype=torch.float64, device="cuda")
    gather = None
    if world > 1:
        from paper_1308_2066_gb300.sharding import gather_ylt
        gather = gather_ylt

    paths = [prec] + ([] if args.no_variants else [p for p in (0, 2, 1) if p != prec])
    tuned = {}
    if not args.no_tune:
        for p in paths:
            tuned[PRECISION_NAMES[p]] = are.are_autotune(ctx, [res.layer], res.yet, p, stream)
    results = {}
    for p in paths:
        r = time_path(are, torch, res, p, args.steps, args.warmup, stream, ylt, gather, world)
        r["ms"] = max_over_ranks(r["ms"], world, torch)
        r["sim_ms"] = max_over_ranks(r["sim_ms"], world, torch)
        results[p] = r
    folded = None
    if not args.no_variants:
        folded = time_folded(are, torch, res, args.steps, args.warmup, stream, ylt, gather, world)
        folded["ms"] = max_over_ranks(folded["ms"], world, torch)
        folded["sim_ms"] = max_over_ranks(folded["sim_ms"], world, torch)
    # the gather ceiling for each row size timed (same YET, no arithmetic)
    ceilings, rows = {}, {}
    for p in paths:
        rows[p] = layer_rows(are, ctx, res.layer, res.yet, p, tuned.get(PRECISION_NAMES[p]))
        rb = rows[p][0]
        if rb not in ceilings:
            ceilings[rb] = are.are_gather_ceiling(ctx, res.yet, rb, 0, y.n_trials, reps=3,
                                                  shapes=True)

    head = results[prec]
    lookups = world * y.n_events * J
    ms_step = head["ms"] / args.steps
    line = {
        "metric": METRIC,
        "value": round(lookups / (ms_step * 1e-3) / 1e9, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "sim_time_s": round(head["sim_ms"] * 1e-3, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[prec],
        "data": "synthetic: seeded uniform YET ids, lognormal(11,1.5) ELT losses (paper's data is proprietary)",
        "config": {"workload": wl.name, "trials_per_gpu": y.n_trials, "events_per_trial": y.k,
                   "elts": J, "catalog": y.catalog, "precision": PRECISION_NAMES[prec],
                   "step": ("repack table + simulate all trials + PML 100/250 + TVaR 99 into device "
                            "arrays + their copy to pinned host memory; steps queued back to back"),
                   "l2": "inputs larger than L2 (4 GB YET streamed every step)",
                   "parallelism": f"trial blocks per GPU x{world}",
                   "gpu": torch.cuda.get_device_name()},
        "roofline": roofline(y.n_events, y.n_trials, J, prec, head["sim_ms"],
                             tuned.get(PRECISION_NAMES[prec]), ceilings[rows[prec][0]], rows[prec]),
        "tuned": tuned,
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "pml": head["pml"], "tvar": head["tvar"],
    }
    line["variants"] = {
        PRECISION_NAMES[p]: {"ms_per_step": round(r["ms"] / args.steps, 4),
                             "sim_ms": round(r["sim_ms"], 4),
                             "value": round(lookups / (r["ms"] / args.steps * 1e-3) / 1e9, 3),
                             "roofline": roofline(y.n_events, y.n_trials, J, p, r["sim_ms"],
                                                  tuned.get(PRECISION_NAMES[p]), ceilings[rows[p][0]],
                                                  rows[p]),
                             "pml": r["pml"], "tvar": r["tvar"], "clocks": r["clocks"]}
        for p, r in results.items() if p != prec}
    if folded is not None:
        ms_f = folded["ms"] / args.steps
        line["variants"]["fp64_folded"] = {
            "what": ("one lookup per occurrence: the layer's FP64 occurrence loss per catalog "
                     "event, built every step, then exact per-trial sums; not the per-ELT "
                     "lookups of the headline"),
            "ms_per_step": round(ms_f, 4), "sim_ms": round(folded["sim_ms"], 4),
            "value": round(lookups / (ms_f * 1e-3) / 1e9, 3),
            "value_unit": "G event-ELT lookups/s equivalent (events x J / step time)",
            "events_per_s": round(world * y.n_events / (ms_f * 1e-3), 1),
            "roofline": folded_roofline(y.n_events, y.n_trials, folded["sim_ms"]),
            "pml": folded["pml"], "tvar": folded["tvar"], "clocks": folded["clocks"],
            "gpu_launches": folded["launches"]}

    if not args.no_e2e:
        line["e2e"] = run_e2e(are, torch, ctx, wl, prec, max(1, min(args.steps, 10)), 1, world)

    if world == 1 and not args.no_subrecords and not args.no_variants:
        line["next_rows"] = next_record(are, torch, res, max(3, min(args.steps, 10)), 3)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, cores, dt = oracle_rate(wl, args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(rate / 1e9, 6), "unit": UNIT, "cores": cores,
                                "kind": "oracle",
                                "sample": f"first {n} of the {y.n_trials} trials ({dt:.1f} s wall, "
                                          f"FP64 oracle, all host threads)"}
    are.are_destroy(ctx)
    del res
    torch.cuda.empty_cache()
    if world == 1 and not args.no_subrecords:
        line.update(subrecords(are, torch, args))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
