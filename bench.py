#!/usr/bin/env python
"""Benchmark of the near-field force path on GB300 (one JSON line on stdout).

Step: one forward pass (nf_forces: binning, work list, pair kernel, FP64
combine) plus one adjoint pass (nf_forces_adjoint) over the clustered
128^3 workload (2,097,152 particles, K = 32, R = 2, eps = 1/(40 * 128)),
inputs resident in HBM.  `value` counts the pair interactions the step computes
(P forward + P adjoint, P = sum_c n_c S_c) per second of device time.  L2 is
flushed (a 512 MB write) before every timed step; each step is bracketed by
CUDA events on the launching stream.

Also reported, from the same run:
  roofline      the forward pair kernel against the FP32 peak (23 flop per pair)
  bin_roofline  the binning stage against the measured HBM copy bandwidth
  e2e           the same step through the public API from pinned host buffers
  batched       64 boxes (the batched recipe) in one captured CUDA graph
  error         fractional force error of this run's output on the oracle sample
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample of sinks

With --gpus N > 1 (torchrun, one rank per GPU) every rank runs its own box
(seed offset by rank): weak scaling, no data-path communication.
`--impl reference` times the FP64 CPU oracle as it stands instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "near-field pair-interactions/s on 1 GB300: fwd, fwd+adjoint, batched; at stated error"
UNIT = "pair-interactions/s"
FLOP_PER_PAIR = 23  # convention fixed for this metric (the paper quotes ~26 incl. rsqrt)
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="clustered", choices=["plain", "clustered", "large", "adjoint"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", default=None, help="sinks_per_lane,stage,warps,blocks_per_sm")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, rank: int):
    import workloads as W
    if name == "plain":
        w = W.config_plain(seed=0 + 1000 * rank)
    elif name == "clustered":
        w = W.config_clustered(seed=1 + 1000 * rank)
    elif name == "large":
        w = W.config_large(seed=2 + 1000 * rank)
    else:
        w = W.config_adjoint(seed=3 + 1000 * rank)
    g = W.upstream_gradient(w.N, 33 + 1000 * rank)
    return w, g


def describe(w) -> str:
    return (f"{w.name}: N={w.N} {'clustered recipe' if w.name != 'plain' else 'uniform'}, "
            f"K={w.K}, R={w.R}, eps={w.eps:.6g} (Plummer-equivalent), unit box")


# ---------------------------------------------------------------------------
# pair counts (measurement only: P = sum_c n_c S_c from cell occupancies)
# ---------------------------------------------------------------------------

def stencil_sums(counts: np.ndarray, R: int) -> np.ndarray:
    """S_c = sum of occupancies over the (2R+1)^3 cells around every cell."""
    S = np.zeros_like(counts, dtype=np.int64)
    c64 = counts.astype(np.int64)
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for c in range(-R, R + 1):
                S += np.roll(c64, (a, b, c), axis=(0, 1, 2))
    return S


# ---------------------------------------------------------------------------
# ranks (one box per GPU; the only collectives are timing and the barrier)
# ---------------------------------------------------------------------------

def aggregate_over_ranks(pairs_local: float, t_local: float, device) -> tuple:
    """Whole-job throughput: pair interactions summed over ranks / the slowest
    rank's time.  Returns (value, t_max, pairs_total)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return pairs_local / t_local, t_local, pairs_local
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([pairs_local], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(p.item()) / float(t.item()), float(t.item()), float(p.item())


def shard_boxes(boxes, rank: int, world: int):
    """Round-robin share of independent boxes for one rank (no communication)."""
    return [b for i, b in enumerate(boxes) if i % world == rank]


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.out = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.bus_id:
                cmd += ["-i", self.bus_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # several GPUs visible to nvidia-smi: keep the one that drew the most power
        by_gpu = {}
        for r in rows:
            by_gpu.setdefault(r[0].strip(), []).append(r)

        def mean_power(rs):
            v = [float(r[4]) for r in rs if r[4].strip() not in ("[N/A]", "N/A")]
            return float(np.mean(v)) if v else 0.0

        rows = max(by_gpu.values(), key=mean_power)
        sm = [float(r[2]) for r in rows]
        mx = max(float(r[3]) for r in rows)
        power = [float(r[4]) for r in rows if r[4].strip() not in ("[N/A]", "N/A")]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].strip() == "Active"})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# oracle CPU baseline (test infrastructure, host cores)
# ---------------------------------------------------------------------------

def oracle_sample(w, g, seconds: float, seed: int = 22):
    """Time the FP64 oracle (forces + adjoint) on a random sample of sinks sized
    to about `seconds` of host work.  Returns (stats dict, sinks, acc_ref)."""
    import oracle
    off, _, _ = oracle.bin_particles(w.pos, w.box, w.K)
    counts = np.diff(off).reshape(w.K, w.K, w.K)
    S = stencil_sums(counts, w.R).reshape(-1)
    cid = oracle.cell_of(w.pos, w.box, w.K)
    rng = np.random.default_rng(seed)
    order = rng.permutation(w.N)
    g64 = g.astype(np.float64)

    def run(n):
        sk = np.sort(order[:n])
        t0 = time.perf_counter()
        oracle.forces(w.pos, w.box, w.K, w.R, w.eps, sinks=sk)
        oracle.adjoint(w.pos, g64, w.box, w.K, w.R, w.eps, sinks=sk)
        return time.perf_counter() - t0

    # calibrate t(n) = a + b n on two small samples (a: the oracle's own binning per call)
    n0, n1 = min(w.N, 128), min(w.N, 1024)
    t0, t1 = run(n0), run(n1)
    b = max((t1 - t0) / max(n1 - n0, 1), 1e-9)
    a = max(t0 - b * n0, 0.0)
    n = int(min(w.N, max(n1, (seconds - a) / b)))
    sinks = np.sort(order[:n])
    t0 = time.perf_counter()
    acc_ref = oracle.forces(w.pos, w.box, w.K, w.R, w.eps, sinks=sinks)
    oracle.adjoint(w.pos, g64, w.box, w.K, w.R, w.eps, sinks=sinks)
    dt = time.perf_counter() - t0
    pairs = 2 * int(S[cid[sinks]].sum())
    cores = oracle.num_threads()
    # the same oracle on one host core, on a smaller sample (about 3 s)
    n1c = int(min(n, max(16, 3.0 / (b * max(cores, 1)))))
    sk1 = np.sort(order[n:n + n1c]) if n + n1c <= w.N else np.sort(order[:n1c])
    t0 = time.perf_counter()
    oracle.forces(w.pos, w.box, w.K, w.R, w.eps, sinks=sk1, threads=1)
    oracle.adjoint(w.pos, g64, w.box, w.K, w.R, w.eps, sinks=sk1, threads=1)
    dt1 = time.perf_counter() - t0
    pairs1 = 2 * int(S[cid[sk1]].sum())
    return ({"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"forces + adjoint for {n} random sinks (seed {seed}) of {w.N}; "
                       f"{pairs:.3e} pair interactions in {dt:.1f} s, FP64, OpenMP",
             "one_core": {"value": pairs1 / dt1, "unit": UNIT, "cores": 1,
                          "sample": f"forces + adjoint for {n1c} random sinks; "
                                    f"{pairs1:.3e} pair interactions in {dt1:.1f} s, including the "
                                    f"oracle's per-call binning of all {w.N} particles"}},
            sinks, acc_ref)


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------

def run_native(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if args.tune:
        _lib.nf_set_default_tuning(tuple(int(x) for x in args.tune.split(",")))

    w, g_np = make_workload(args.workload, rank)
    N = w.N
    pos = torch.from_numpy(w.pos).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    ws = torch.empty(_lib.nf_workspace_bytes(N, w.K, w.R), dtype=torch.uint8, device=dev)
    acc = torch.empty_like(pos)
    grad = torch.empty_like(pos)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
        _lib.nf_forces_adjoint(pos, g, w.box, w.K, w.R, w.eps, grad, ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = _lib.nf_stats_read(ws)
    P = st["pairs"]

    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id  # type: ignore[attr-defined]
    except Exception:
        bus = None
    clocks = ClockSampler(bus if isinstance(bus, str) else None)

    # ---- timed region: device time of exactly K steps, L2 flushed before each
    _lib.nf_profile_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    prof_fwd, prof_adj = [], []
    launches0 = _lib.nf_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        prof_fwd.append(_lib.nf_profile_read(1))
        prof_adj.append(_lib.nf_profile_read(0))
    torch.cuda.synchronize()
    launches = _lib.nf_kernel_launches() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    _lib.nf_profile_enable(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    value, t_max, pairs_all = aggregate_over_ranks(2 * P * args.steps, t_total, dev)

    fwd_pair_ms = float(np.mean([p["pair_ms"] for p in prof_fwd]))
    adj_pair_ms = float(np.mean([p["pair_ms"] for p in prof_adj]))
    fwd_ms = float(np.mean([p["total_ms"] for p in prof_fwd]))
    adj_ms = float(np.mean([p["total_ms"] for p in prof_adj]))
    bin_ms = float(np.mean([p["bin_ms"] for p in prof_fwd]))

    # ---- roofline of the forward pair kernel (FP32 issue-bound: "alu")
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    max_mhz = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s, 128 FP32 lanes/SM, FMA = 2 flop
    achieved = FLOP_PER_PAIR * P / (fwd_pair_ms / 1e3) / 1e12
    fma = measure_fma_peak(dev)
    traffic = kernel_traffic("force", args.workload)
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic,
                "kernel": "k_force (forward pair loop)",
                "peak_basis": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {max_mhz:.0f} MHz max SM clock",
                "frac_at_sampled_clock": (achieved / (sms * 256 * clk["sm_mhz"] * 1e6 / 1e12)
                                          if clk.get("sm_mhz") else None),
                "flop_per_pair": FLOP_PER_PAIR,
                "measured_fma_peak": fma,
                "frac_of_measured_fma": achieved / max(fma["scalar_tflops"], fma["packed_tflops"])}
    hbm = peaks.get("hbm_gbs", 6786.2)
    bin_bytes = 32.0 * N + 8.0 * (w.K ** 3 + 1)
    bin_roof = {"bound": "hbm", "achieved": bin_bytes / (bin_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bin_bytes / (bin_ms / 1e3) / 1e9 / hbm, "traffic": kernel_traffic("bin", args.workload),
                "bytes_per_particle": 32, "note": "algorithmic bytes: pos 12 + rel 16 + perm 4 per particle + offsets"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(w), "pairs_per_pass": P, "pairs_per_step": 2 * P,
                   "step": "nf_forces + nf_forces_adjoint", "l2": "flushed (512 MB write) before each step",
                   "parallelism": f"replicas: one box per GPU x {world}",
                   "tuning": list(_lib.nf_get_default_tuning())},
        "fwd": {"pairs_per_s": P / (fwd_ms / 1e3), "particle_updates_per_s": N / (fwd_ms / 1e3),
                "ms": fwd_ms, "pair_kernel_ms": fwd_pair_ms, "bin_ms": bin_ms},
        "fwd_adjoint": {"pairs_per_s": P / ((fwd_ms + adj_ms) / 1e3), "ms": fwd_ms + adj_ms,
                        "adjoint_pair_kernel_ms": adj_pair_ms, "over_fwd": (fwd_ms + adj_ms) / fwd_ms},
        "roofline": roofline, "bin_roofline": bin_roof,
        "gpu_launches": int(launches), "clocks": clk,
        "stats": {"max_cell_occupancy": st["max_occupancy"], "work_items": st["items"],
                  "lane_utilisation": st["pairs"] / max(st["lane_pairs"], 1)},
    }

    out["uniform"] = measure_uniform(w, dev, flush, fp32_peak)
    out["density"] = measure_density(w, pos, ws, acc, fwd_pair_ms, flush)
    out["kdk"] = measure_kdk(w, dev, flush)
    out["multipoles"] = measure_multipoles(w, pos, dev, flush)
    out["far"] = measure_far(w, pos, dev, flush, fma, fwd_ms_for_far(out))
    if not args.no_e2e:
        out["e2e"] = measure_e2e(args, w, g_np, dev, P, flush)
    if not args.no_batched:
        out["batched"] = measure_batched(dev, flush, rank, world)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cb, sinks, ref = oracle_sample(w, g_np, args.cpu_seconds)
        out["cpu_baseline"] = cb
        import oracle
        a = acc.cpu().numpy()[sinks]
        e = oracle.frac_error(a, ref)
        out["error"] = {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)),
                        "max": float(e.max()), "sample": int(len(sinks)),
                        "bar": {"median": 1e-6, "max": 1e-4}}
    elif rank == 0:
        out["cpu_baseline"] = None
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def measure_fma_peak(dev, target_ms=40.0, reps=3):
    """FP32 multiply-add throughput of this GPU (nf_fma_probe), scalar and packed
    f32x2, timed with events on the launching stream: the measured denominator
    beside the derived FP32 peak."""
    import torch
    from paper_2110_11392_gb300 import _lib
    sink = torch.empty(_lib.nf_fma_probe_sink_floats(), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev)
    out = {}
    for mode in (0, 1, 2):
        def timed(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            flop = _lib.nf_fma_probe(sink, iters, mode, s)
            e1.record(s)
            e1.synchronize()
            return flop, e0.elapsed_time(e1)
        timed(256)
        flop, ms = timed(2048)
        iters = int(min(1 << 24, max(2048, 2048 * target_ms / max(ms, 1e-3))))
        best = 0.0
        for _ in range(reps):
            flop, ms = timed(iters)
            best = max(best, flop / (ms / 1e3) / 1e12)
        out[("scalar_tflops", "packed_tflops", "fp64_tflops")[mode]] = best
    out["unit"] = "TFLOP/s"
    out["probe"] = ("nf_fma_probe: 4 x 256 threads per SM, 8 independent multiply-add chains per thread "
                    "(f32, f32x2, f64), best of 3")
    return out


def measure_uniform(w, dev, flush, fp32_peak, reps=5):
    """The forward on a uniform (i.i.d.) set of the same N, K, R and softening
    as the workload (seed 101): pair kernel and whole call, pairs/s and the
    fraction of the FP32 roofline."""
    import torch
    import workloads as W
    from paper_2110_11392_gb300 import _lib
    pos = torch.from_numpy(W.uniform_positions(w.N, 101, w.box)).to(dev)
    ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device=dev)
    acc = torch.empty_like(pos)
    _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
    P = _lib.nf_stats_read(ws)["pairs"]
    stream = torch.cuda.current_stream(dev)
    _lib.nf_profile_enable(True)
    call_ms, pair_ms = [], []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
        b.record(stream)
        b.synchronize()
        call_ms.append(a.elapsed_time(b))
        pair_ms.append(_lib.nf_profile_read(0)["pair_ms"])
    _lib.nf_profile_enable(False)
    t_call, t_pair = float(np.median(call_ms)), float(np.median(pair_ms))
    achieved = FLOP_PER_PAIR * P / (t_pair / 1e3) / 1e12
    return {"workload": f"uniform: N={w.N}, K={w.K}, R={w.R}, same softening, seed 101", "pairs_per_pass": P,
            "pair_kernel_ms": t_pair, "ms": t_call, "pairs_per_s": P / (t_call / 1e3),
            "pair_kernel_pairs_per_s": P / (t_pair / 1e3),
            "particle_updates_per_s": w.N / (t_call / 1e3), "roofline_frac": achieved / fp32_peak}


def measure_density(w, pos, ws, acc, fwd_pair_ms, flush):
    """The forward with the fused top-hat density estimate (b = half a cell):
    its pair kernel time against the plain forward pair kernel."""
    import torch
    from paper_2110_11392_gb300 import _lib
    b = 0.5 * w.box / w.K
    rho = torch.empty(w.N, dtype=torch.float32, device=pos.device)
    _lib.nf_forces_density(pos, w.box, w.K, w.R, w.eps, b, acc, rho, ws)
    _lib.nf_profile_enable(True)
    ms = []
    for _ in range(3):
        flush.zero_()
        _lib.nf_forces_density(pos, w.box, w.K, w.R, w.eps, b, acc, rho, ws)
        ms.append(_lib.nf_profile_read(0)["pair_ms"])
    _lib.nf_profile_enable(False)
    t = float(np.mean(ms))
    return {"b_cells": 0.5, "pair_kernel_ms": t, "over_fwd_pair_kernel": t / fwd_pair_ms,
            "mean_rho": float(rho.mean().item())}


def measure_kdk(w, dev, flush, steps=5):
    """Leapfrog steps with the adaptive global time step, all on the device:
    kick, drift, near-field forces, kick and Eq. (timestep) per step."""
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    rng = np.random.default_rng(9)
    pos = torch.from_numpy(w.pos).to(dev)
    vel = torch.from_numpy((0.01 * rng.standard_normal((w.N, 3))).astype(np.float32)).to(dev)
    ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device=dev)
    acc = nf.forces(pos, w.box, w.K, w.R, w.eps, ws=ws)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    prm = _lib.make_step_params(0.25)
    _lib.nf_timestep(pos, vel, acc, w.box, w.K, prm, dt, ws)
    stream = torch.cuda.current_stream(dev)
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.nf_kdk_step(pos, vel, acc, w.box, w.K, w.R, w.eps, dt, prm, ws)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.mean(ms))
    return {"ms_per_step": t, "particle_updates_per_s": w.N / (t / 1e3), "last_dt": float(dt.item()),
            "steps": steps, "note": "kick + drift + nf_forces + kick + Eq. (timestep), near field only"}


def fwd_ms_for_far(out):
    return out["fwd"]["ms"]


def taylor_flop_per_particle(p: int) -> int:
    """FP64 flops of the nested Horner evaluation of the Taylor series and its
    gradient at one particle: 2 multiply-adds per term (z), 3 per (a, b) (y),
    4 per a (x); 2 flops each."""
    nt = (p + 3) * (p + 2) * (p + 1) // 6
    nab = (p + 2) * (p + 1) // 2
    return 2 * (2 * nt + 3 * nab + 4 * (p + 1))


def taylor_df_ops_per_particle(p: int) -> int:
    """FP32 instructions of the double-float Taylor evaluation at one particle:
    the Horner steps of taylor_flop_per_particle, 11 FP32 instructions each
    (product with its FMA error terms, TwoSum, two adds; the steps skip the
    renormalisation)."""
    nt = (p + 3) * (p + 2) * (p + 1) // 6
    nab = (p + 2) * (p + 1) // 2
    return 11 * (2 * nt + 3 * nab + 4 * (p + 1))


def measure_far(w, pos, dev, flush, fma, fwd_ms, p=8, reps=5):
    """The far field at order p on the same particles: derivatives once, then
    nf_far_forces per call (binning, multipoles, FFT convolution, Taylors);
    the total force of a user's step (nf_forces_total: near + far, one
    binning); and leapfrog steps with that force (nf_kdk_step_far)."""
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    a, b = ev(), ev()
    torch.cuda.synchronize(dev)
    ff = nf.FarField(w.K, w.R, p, w.box, device=dev)   # first call: allocations and cuFFT plans
    ws = ff.workspace(w.N)
    torch.cuda.synchronize(dev)
    a.record(stream)
    _lib.nf_derivatives(w.K, w.R, p, w.box, ff.derivs, ws)  # the precompute alone, on the device
    b.record(stream)
    b.synchronize()
    deriv_ms = a.elapsed_time(b)
    acc = torch.empty((w.N, 3), dtype=torch.float64, device=dev)
    wsn = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device=dev)
    tot = torch.empty((w.N, 3), dtype=torch.float32, device=dev)
    def far_call_ms():
        for _ in range(2):
            _lib.nf_far_forces(pos, w.box, w.K, w.R, p, ff.derivs, acc, None, None, ws)
        ms = []
        for _ in range(reps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            _lib.nf_far_forces(pos, w.box, w.K, w.R, p, ff.derivs, acc, None, None, ws)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))
    # the other arithmetic of the per-particle kernels, for comparison
    arith = _lib.nf_far_get_arith()
    other = _lib.NF_FAR_FP64 if arith == _lib.NF_FAR_DOUBLE_FLOAT else _lib.NF_FAR_DOUBLE_FLOAT
    _lib.nf_far_set_arith(other)
    other_ms = far_call_ms()
    _lib.nf_far_set_arith(arith)
    for _ in range(2):
        _lib.nf_far_forces(pos, w.box, w.K, w.R, p, ff.derivs, acc, None, None, ws)
    _lib.nf_profile_enable(True)
    far_ms, prof = [], []
    for _ in range(reps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        _lib.nf_far_forces(pos, w.box, w.K, w.R, p, ff.derivs, acc, None, None, ws)
        b.record(stream)
        b.synchronize()
        far_ms.append(a.elapsed_time(b))
        prof.append(_lib.nf_far_profile_read(0))
    _lib.nf_profile_enable(False)
    tot_ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        _lib.nf_forces_total(pos, w.box, w.K, w.R, w.eps, p, ff.derivs, tot, wsn, ws)
        b.record(stream)
        b.synchronize()
        tot_ms.append(a.elapsed_time(b))
    # leapfrog steps with the total force (nf_kdk_step_far, adaptive dt)
    rng = np.random.default_rng(9)
    xs = pos.clone()
    vel = torch.from_numpy((0.01 * rng.standard_normal((w.N, 3))).astype(np.float32)).to(dev)
    acc_t = torch.empty((w.N, 3), dtype=torch.float32, device=dev)
    _lib.nf_forces(xs, w.box, w.K, w.R, w.eps, acc_t, None, wsn)
    _lib.nf_far_forces(xs, w.box, w.K, w.R, p, ff.derivs, None, acc_t, None, ws)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    prm = _lib.make_step_params(0.25)
    _lib.nf_timestep(xs, vel, acc_t, w.box, w.K, prm, dt, wsn)
    step_ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        _lib.nf_kdk_step_far(xs, vel, acc_t, w.box, w.K, w.R, w.eps, p, ff.derivs, dt, prm, wsn, ws)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    stage = {k: float(np.median([q[k] for q in prof])) for k in prof[0]}
    t_ms = float(np.median(far_ms))
    if arith == _lib.NF_FAR_DOUBLE_FLOAT:
        # FP32-pipe bound: instructions per second against the measured scalar FP32 rate
        ops = taylor_df_ops_per_particle(p) * w.N
        achieved = ops / (stage["taylor_ms"] / 1e3) / 1e12
        peak32 = fma["scalar_tflops"] / 2.0  # one FMA = 2 flop = 1 instruction
        taylor_roof = {"bound": "alu", "achieved": achieved, "peak": peak32, "unit": "T FP32 instructions/s",
                       "frac": achieved / peak32, "op_per_particle": taylor_df_ops_per_particle(p),
                       "peak_basis": "measured: nf_fma_probe fma.rn.f32 rate / 2, this run"}
    else:
        flop = taylor_flop_per_particle(p) * w.N
        achieved = flop / (stage["taylor_ms"] / 1e3) / 1e12
        peak64 = fma["fp64_tflops"]
        taylor_roof = {"bound": "fp64", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                       "frac": achieved / peak64, "flop_per_particle": taylor_flop_per_particle(p),
                       "peak_basis": "measured: nf_fma_probe fma.rn.f64, this run"}
    names = {_lib.NF_FAR_FP64: "fp64", _lib.NF_FAR_DOUBLE_FLOAT: "double-float"}
    return {"order": p, "terms": (p + 3) * (p + 2) * (p + 1) // 6, "derivatives_ms": deriv_ms,
            "ms": t_ms, "particles_per_s": w.N / (t_ms / 1e3), "stages_ms": stage,
            "total_force_ms": float(np.median(tot_ms)),
            "total_force_particles_per_s": w.N / (float(np.median(tot_ms)) / 1e3),
            "near_forward_ms": fwd_ms,
            "kdk_total_force_ms_per_step": float(np.median(step_ms)),
            "kdk_total_force_particle_updates_per_s": w.N / (float(np.median(step_ms)) / 1e3),
            "arith": names[arith], "other_arith": {"arith": names[other], "ms": other_ms},
            "taylor_roofline": taylor_roof,
            "note": "derivatives in FP64, once per (K, R, p, box); in double-float mode (K a power of two) the "
                    "multipoles, transforms, k-space product, rebuild and Taylors are double-float on the FP32 "
                    "pipe; in FP64 mode cuFFT and FP64 kernels; Ewald-summed periodic force = near + far"}


def measure_multipoles(w, pos, dev, flush, p=8, reps=3):
    """Complete-basis cell multipoles at order p (FP64): binning + nf_multipoles."""
    import torch
    from paper_2110_11392_gb300 import _lib
    nt = (p + 3) * (p + 2) * (p + 1) // 6
    M = torch.empty((w.K ** 3, nt), dtype=torch.float64, device=dev)
    ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device=dev)
    _lib.nf_multipoles(pos, w.box, w.K, p, M, ws)
    stream = torch.cuda.current_stream(dev)
    ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.nf_multipoles(pos, w.box, w.K, p, M, ws)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.mean(ms)) / 1e3
    flop = w.N * (3 * p + 3 * nt)  # powers, then a multiply and an FMA per term
    return {"order": p, "terms": nt, "ms": t * 1e3, "particles_per_s": w.N / t,
            "fp64_tflops": flop / t / 1e12, "note": "includes binning; FP64 throughout"}


def measure_e2e(args, w, g_np, dev, P, flush):
    """Same step through the public API with pinned host inputs and outputs:
    every step copies its positions and upstream gradient in and its
    accelerations and gradient out.  Pipelined: step i + 1's upload (a
    copy-in stream) and step i's download (a copy-out stream) overlap step
    i's compute, with double-buffered device tensors ordered by events; the
    timed region spans all steps, from the first upload to the last download
    (the L2 flush still runs before every step).  The serial form, one step at
    a time, is reported beside it."""
    import torch
    import paper_2110_11392_gb300 as nf
    hp = torch.from_numpy(w.pos).pin_memory()
    hg = torch.from_numpy(g_np).pin_memory()
    ha = torch.empty_like(hp).pin_memory()
    hgr = torch.empty_like(hp).pin_memory()
    stream = torch.cuda.current_stream(dev)
    cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    dpos = [torch.empty_like(hp, device=dev) for _ in range(2)]
    dg = [torch.empty_like(hp, device=dev) for _ in range(2)]
    dacc = [torch.empty_like(hp, device=dev) for _ in range(2)]
    dgr = [torch.empty_like(hp, device=dev) for _ in range(2)]
    ev = lambda: torch.cuda.Event()

    def serial_step():
        pos = hp.to(dev, non_blocking=True)
        g = hg.to(dev, non_blocking=True)
        acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
        grad = nf.forces_adjoint(pos, g, w.box, w.K, w.R, w.eps)
        ha.copy_(acc, non_blocking=True)
        hgr.copy_(grad, non_blocking=True)

    def pipelined(n):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        in_done, comp_done, out_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        t0.record(stream)
        cin.wait_event(t0)
        with torch.cuda.stream(cin):
            dpos[0].copy_(hp, non_blocking=True)
            dg[0].copy_(hg, non_blocking=True)
            in_done[0].record(cin)
        for i in range(n):
            b = i % 2
            if i + 1 < n:  # next step's upload into the other buffers, once step i-1 is done with them
                with torch.cuda.stream(cin):
                    if i >= 1:
                        cin.wait_event(comp_done[1 - b])
                    dpos[1 - b].copy_(hp, non_blocking=True)
                    dg[1 - b].copy_(hg, non_blocking=True)
                    in_done[1 - b].record(cin)
            stream.wait_event(in_done[b])
            if i >= 2:
                stream.wait_event(out_done[b])  # step i-2's download of these outputs
            flush.zero_()
            nf.forces(dpos[b], w.box, w.K, w.R, w.eps, out=dacc[b])
            nf.forces_adjoint(dpos[b], dg[b], w.box, w.K, w.R, w.eps, out=dgr[b])
            comp_done[b].record(stream)
            with torch.cuda.stream(cout):
                cout.wait_event(comp_done[b])
                ha.copy_(dacc[b], non_blocking=True)
                hgr.copy_(dgr[b], non_blocking=True)
                out_done[b].record(cout)
        stream.wait_event(out_done[(n - 1) % 2])
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / 1e3

    for _ in range(2):
        serial_step()
    pipelined(3)
    torch.cuda.synchronize()
    n = max(3, args.steps // 3)
    tot = 0.0
    for _ in range(n):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        serial_step()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b) / 1e3
    t_pipe = pipelined(n)
    return {"value": 2 * P * n / t_pipe, "unit": UNIT, "h2d_bytes_per_step": 2 * w.pos.nbytes,
            "d2h_bytes_per_step": 2 * w.pos.nbytes, "steps": n,
            "serial_value": 2 * P * n / tot,
            "note": "pinned host pos and g in, acc and grad out, every step; uploads and downloads on "
                    "their own streams overlapping the neighbouring steps' compute (serial_value: one "
                    "step at a time)"}


def measure_batched(dev, flush, rank=0, world=1):
    """64 boxes (batched recipe): one captured graph of nf_forces_batched vs one
    nf_forces call per box.  With several ranks the boxes are shared round-robin
    and the rates are summed (slowest rank's time)."""
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    import workloads as W
    w = W.config_batched()
    rows, off = [], 0
    for b in w.boxes:
        rows.append((off, b))
        off += b["N"]
    mine = shard_boxes(rows, rank, world)
    boxes = [b for _, b in mine]
    pos_np = np.concatenate([w.pos[o:o + b["N"]] for o, b in mine])
    w.boxes = boxes
    w.pos = pos_np
    run = nf.BatchedNearField(w.boxes, device=dev)
    run.pos.copy_(torch.from_numpy(w.pos).to(dev))
    run()
    torch.cuda.synchronize()
    P = run.stats()["pairs"]
    run.capture()
    stream = torch.cuda.current_stream(dev)
    reps = 5

    def timed(fn):
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b) / 1e3
        return tot / reps

    t_graph = timed(lambda: run())
    parts, off = [], 0
    for bx in w.boxes:
        parts.append((run.pos[off:off + bx["N"]], run.acc[off:off + bx["N"]], bx))
        off += bx["N"]
    ws = torch.empty(max(_lib.nf_workspace_bytes(bx["N"], bx["K"], bx["R"]) for bx in w.boxes),
                     dtype=torch.uint8, device=dev)

    def separate():
        for p, a, bx in parts:
            _lib.nf_forces(p, bx["box"], bx["K"], bx["R"], bx["eps"], a, None, ws)

    separate()
    t_sep = timed(separate)
    rate_g, t_graph, P_all = aggregate_over_ranks(float(P), t_graph, dev)
    rate_s, t_sep, _ = aggregate_over_ranks(float(P), t_sep, dev)
    return {"pairs_per_s": rate_g, "separate_pairs_per_s": rate_s, "speedup": t_sep / t_graph,
            "boxes": 64, "boxes_per_rank": len(w.boxes), "pairs": P_all, "graph_ms": t_graph * 1e3,
            "separate_ms": t_sep * 1e3}


def kernel_traffic(which: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary of this workload, if it matches the current source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[workload][which]
    except (OSError, ValueError, KeyError, TypeError):
        return None
    src = os.path.join(ROOT, "paper_2110_11392_gb300", "csrc", rec.get("source", ""))
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec.get("bytes_per_launch") if h == rec.get("sha256_16") else None


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle as it stands, on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    w, g_np = make_workload(args.workload, 0)
    budget = max(2.0, 150.0 / (args.steps + args.warmup))
    # one calibration sample fixes the per-step sample size
    cb, sinks, _ = oracle_sample(w, g_np, budget)
    g64 = g_np.astype(np.float64)
    off, _, _ = oracle.bin_particles(w.pos, w.box, w.K)
    S = stencil_sums(np.diff(off).reshape(w.K, w.K, w.K), w.R).reshape(-1)
    cid = oracle.cell_of(w.pos, w.box, w.K)
    n = len(sinks)
    rng = np.random.default_rng(23)
    times, pairs = [], []
    for k in range(args.warmup + args.steps):
        sk = np.sort(rng.choice(w.N, n, replace=False))
        t0 = time.perf_counter()
        oracle.forces(w.pos, w.box, w.K, w.R, w.eps, sinks=sk)
        oracle.adjoint(w.pos, g64, w.box, w.K, w.R, w.eps, sinks=sk)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            pairs.append(2 * int(S[cid[sk]].sum()))
    value = sum(pairs) / sum(times)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": describe(w), "step": f"oracle forces + adjoint on {n} random sinks"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{n} random sinks of {w.N} per step, forces + adjoint, FP64"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world, local)


if __name__ == "__main__":
    main()
