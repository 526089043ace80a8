#!/usr/bin/env python
"""Benchmark of the near-field force path on GB300 (one JSON line on stdout).

Step: one forward pass (nf_forces: binning, work list, pair kernel,
combine) plus one adjoint pass (nf_forces_adjoint) over the large clustered
box (512^3 = 134,217,728 particles, K = 128, R = 2, eps = 1/(40 * 512)),
inputs resident in HBM; `--workload` picks another box (the clustered 128^3
box is also timed beside it, key `clustered128`).  `value` counts the pair interactions the step computes
(P forward + P adjoint, P = sum_c n_c S_c) per second of device time.  L2 is
flushed (a 512 MB write) before every timed step; each step is bracketed by
CUDA events on the launching stream.

Also reported, from the same run:
  roofline      the forward pair kernel against the FP32 peak (23 flop per pair)
  bin_roofline  the binning stage against the measured HBM copy bandwidth
  e2e           the same step through the public API from pinned host buffers
  batched       64 boxes (the batched recipe) in one captured CUDA graph
  error         fractional force error of this run's output on the oracle sample
                (every particle of a fixed random 1 % of the sink cells, seed 22)
  cpu_baseline  the FP64 oracle on the host cores on that sample, its time
                extrapolated to the whole box by the pair-count ratio

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
    ap.add_argument("--workload", default="large",
                    choices=["plain", "clustered", "medium", "medium128", "large", "adjoint"],
                    help="large: the 512^3 box (default); medium: the same recipe at 256^3, K = 64 (for "
                         "profiling at sizes beyond L2); medium128: 256^3 at K = 128 (the binning of the "
                         "512^3 box: three sort passes); clustered: 128^3; adjoint: 64^3; plain: 32^3 uniform")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the secondary measurements (other workloads, density, steps, far field)")
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
    elif name == "medium":
        w = W.config_large(N=256 ** 3, K=64, seed=2 + 1000 * rank)
    elif name == "medium128":
        w = W.config_large(N=256 ** 3, K=128, seed=2 + 1000 * rank)
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

def sample_cells(off: np.ndarray, perm: np.ndarray, frac: float, seed: int = 22):
    """A fixed random sample of sink cells (a fraction `frac` of all cells, seed
    `seed`) and the particles in them, listed cell by cell (the oracle then
    visits the same neighbour cells for consecutive sinks, which keeps its
    memory accesses local; the sums do not depend on the order)."""
    C = off.shape[0] - 1
    counts = np.diff(off)
    rng = np.random.default_rng(seed)
    cells = np.sort(rng.choice(C, max(1, int(round(frac * C))), replace=False))
    mask = np.zeros(C, bool)
    mask[cells] = True
    sinks = perm[np.repeat(mask, counts)].astype(np.int64)
    return cells, sinks


def oracle_sample(w, g, frac: float = 0.01, seed: int = 22, one_core_s: float = 3.0):
    """The FP64 oracle on a fixed random sample of 1 % of the sink cells (seed 22):
    forces and adjoint of every particle in those cells, timed on the host
    cores.  The particle set is binned once (oracle.Grid, the set-up the one-shot
    oracle functions repeat per call; its time is reported beside the rate).
    Returns (stats dict, sinks, acc_ref)."""
    import oracle
    t0 = time.perf_counter()
    grid = oracle.Grid(w.pos, w.box, w.K, w.R, w.eps)
    setup_s = time.perf_counter() - t0
    off, perm = grid.binning()
    counts = np.diff(off)
    S = stencil_sums(counts.reshape(w.K, w.K, w.K), w.R).reshape(-1)
    cells, sinks = sample_cells(off, perm, frac, seed)
    pairs_fwd = int((counts[cells].astype(np.int64) * S[cells]).sum())
    P_full = int((counts.astype(np.int64) * S).sum())
    g64 = g.astype(np.float64)
    t0 = time.perf_counter()
    acc_ref = grid.forces(sinks)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    grid.adjoint(g64, sinks)
    t_adj = time.perf_counter() - t0
    dt = t_fwd + t_adj
    pairs = 2 * pairs_fwd
    cores = oracle.num_threads()
    # the same oracle on one host core, on the first sampled cells (about one_core_s)
    rate1 = pairs / dt / max(cores, 1)
    want = one_core_s * rate1 / 2
    csum = np.cumsum(counts[cells].astype(np.int64) * S[cells])
    nc = int(min(len(cells), max(1, np.searchsorted(csum, want) + 1)))
    m1 = np.zeros(w.K ** 3, bool)
    m1[cells[:nc]] = True
    sk1 = perm[np.repeat(m1, counts)].astype(np.int64)
    t0 = time.perf_counter()
    grid.forces(sk1, threads=1)
    grid.adjoint(g64, sk1, threads=1)
    dt1 = time.perf_counter() - t0
    pairs1 = 2 * int(csum[nc - 1])
    grid.close()
    return ({"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"forces + adjoint of all {len(sinks)} particles (listed cell by cell) in a fixed random 1 % of the sink cells "
                       f"({len(cells)} of {w.K ** 3}, seed {seed}); {pairs:.4e} pair interactions in {dt:.1f} s "
                       f"(forces {t_fwd:.1f} s, adjoint {t_adj:.1f} s), FP64, OpenMP; binning once before "
                       f"({setup_s:.1f} s, not in the rate)",
             "extrapolated": {"full_step_s": dt * (2 * P_full) / pairs, "pairs_per_step": 2 * P_full,
                              "note": "extrapolated: the sample's time scaled by the exact pair-count ratio "
                                      "of the whole box to the sample"},
             "setup_s": setup_s,
             "one_core": {"value": pairs1 / dt1, "unit": UNIT, "cores": 1,
                          "sample": f"forces + adjoint of the {len(sk1)} particles in the first {nc} sampled "
                                    f"cells; {pairs1:.3e} pair interactions in {dt1:.1f} s"}},
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
    bin_traffic = kernel_traffic("bin", args.workload)
    bin_roof = {"bound": "hbm", "achieved": bin_bytes / (bin_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bin_bytes / (bin_ms / 1e3) / 1e9 / hbm, "traffic": bin_traffic,
                "traffic_gbs": bin_traffic / (bin_ms / 1e3) / 1e9 if bin_traffic else None,
                "bytes_per_particle": 32, "note": "algorithmic bytes: pos 12 + rel 16 + perm 4 per particle + offsets; "
                "traffic_gbs: the ncu DRAM bytes of one call over its event time"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(w), "pairs_per_pass": P, "pairs_per_step": 2 * P,
                   "step": "nf_forces + nf_forces_adjoint", "l2": "flushed (512 MB write) before each step",
                   "parallelism": f"replicas: one box per GPU x {world}",
                   "tuning": {"forward": list(_lib.nf_get_default_tuning()),
                              "adjoint": list(_lib.nf_get_default_tuning_adjoint()),
                              "fields": "sinks per lane, sources per stage, warps per block, blocks per SM (0: as many as fit)"}},
        "fwd": {"pairs_per_s": P / (fwd_ms / 1e3), "particle_updates_per_s": N / (fwd_ms / 1e3),
                "ms": fwd_ms, "pair_kernel_ms": fwd_pair_ms, "bin_ms": bin_ms},
        "fwd_adjoint": {"pairs_per_s": P / ((fwd_ms + adj_ms) / 1e3), "ms": fwd_ms + adj_ms,
                        "adjoint_pair_kernel_ms": adj_pair_ms, "over_fwd": (fwd_ms + adj_ms) / fwd_ms},
        "roofline": roofline, "bin_roofline": bin_roof,
        "gpu_launches": int(launches), "clocks": clk,
        "stats": {"max_cell_occupancy": st["max_occupancy"], "work_items": st["items"],
                  "lane_utilisation": st["pairs"] / max(st["lane_pairs"], 1)},
    }

    if not args.no_side:
        if args.workload != "clustered":
            out["clustered128"] = measure_step_side("clustered", dev, flush, fp32_peak, rank)
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
        a_all = acc.cpu().numpy()
        cb, sinks, ref = oracle_sample(w, g_np)
        out["cpu_baseline"] = cb
        import oracle
        e = oracle.frac_error(a_all[sinks], ref)
        out["error"] = {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)),
                        "max": float(e.max()), "sample": int(len(sinks)),
                        "sample_kind": "every particle of a fixed random 1 % of the sink cells (seed 22)",
                        "bar": {"median": 1e-6, "max": 1e-4}}
    elif rank == 0:
        out["cpu_baseline"] = None
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def measure_fma_peak(dev, target_ms=40.0, reps=3):
    """FP32 multiply-add throughput of this GPU (the probe library), scalar and packed
    f32x2, timed with events on the launching stream: the measured denominator
    beside the derived FP32 peak."""
    import torch
    from paper_2110_11392_gb300 import probe
    sink = torch.empty(probe.sink_floats(), dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev)
    out = {}
    for mode in (0, 1, 2):
        def timed(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            flop = probe.fma_probe(sink, iters, mode, s)
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
    out["probe"] = ("libnf_probe.so (the benchmark's own probe, not part of libnf): 4 x 256 threads per SM, 8 independent multiply-add chains per thread "
                    "(f32, f32x2, f64), best of 3")
    return out


def measure_step_side(name, dev, flush, fp32_peak, rank=0, reps=10):
    """The benchmark step (nf_forces + nf_forces_adjoint) on another workload
    (the clustered 128^3 box): rate, call and pair-kernel times, roofline."""
    import torch
    from paper_2110_11392_gb300 import _lib
    w, g_np = make_workload(name, rank)
    pos = torch.from_numpy(w.pos).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device=dev)
    acc = torch.empty_like(pos)
    grad = torch.empty_like(pos)
    stream = torch.cuda.current_stream(dev)

    def step():
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
        _lib.nf_forces_adjoint(pos, g, w.box, w.K, w.R, w.eps, grad, ws)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    P = _lib.nf_stats_read(ws)["pairs"]
    _lib.nf_profile_enable(True)
    ms, pf, pa = [], [], []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        pf.append(_lib.nf_profile_read(1))
        pa.append(_lib.nf_profile_read(0))
    _lib.nf_profile_enable(False)
    t = float(np.mean(ms))
    fwd_pair = float(np.mean([q["pair_ms"] for q in pf]))
    fwd = float(np.mean([q["total_ms"] for q in pf]))
    adj = float(np.mean([q["total_ms"] for q in pa]))
    return {"workload": describe(w), "pairs_per_pass": P, "value": 2 * P / (t / 1e3), "unit": UNIT,
            "ms_per_step": t, "fwd_ms": fwd, "adjoint_ms": adj, "fwd_pair_kernel_ms": fwd_pair,
            "adjoint_pair_kernel_ms": float(np.mean([q["pair_ms"] for q in pa])),
            "bin_ms": float(np.mean([q["bin_ms"] for q in pf])),
            "fwd_adjoint_over_fwd": (fwd + adj) / fwd,
            "roofline_frac": FLOP_PER_PAIR * P / (fwd_pair / 1e3) / 1e12 / fp32_peak}


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
    """The forward with the fused top-hat density estimate: its pair kernel
    time against the plain forward pair kernel, at the FoF scale the paper
    uses it for (b = 0.2 mean interparticle spacings, Sec. "Group Finding")
    and at b = half a cell."""
    import torch
    from paper_2110_11392_gb300 import _lib
    rho = torch.empty(w.N, dtype=torch.float32, device=pos.device)
    spacing = w.box / w.N ** (1.0 / 3.0)
    out = {}
    for name, b in (("fof", 0.2 * spacing), ("half_cell", 0.5 * w.box / w.K)):
        _lib.nf_forces_density(pos, w.box, w.K, w.R, w.eps, b, acc, rho, ws)
        _lib.nf_profile_enable(True)
        ms = []
        for _ in range(3):
            flush.zero_()
            _lib.nf_forces_density(pos, w.box, w.K, w.R, w.eps, b, acc, rho, ws)
            ms.append(_lib.nf_profile_read(0)["pair_ms"])
        _lib.nf_profile_enable(False)
        t = float(np.mean(ms))
        out[name] = {"b_cells": b * w.K / w.box, "pair_kernel_ms": t, "over_fwd_pair_kernel": t / fwd_pair_ms,
                     "mean_rho": float(rho.mean().item())}
    out["note"] = "b = 0.2 mean spacings (FoF scale) and b = half a cell; plain forward pair kernel as the base"
    return out


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
    ff = nf.FarField(w.K, w.R, p, w.box, device=dev)   # first call: allocations
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
                       "peak_basis": "measured: the probe's fma.rn.f32 rate / 2, this run"}
    else:
        flop = taylor_flop_per_particle(p) * w.N
        achieved = flop / (stage["taylor_ms"] / 1e3) / 1e12
        peak64 = fma["fp64_tflops"]
        taylor_roof = {"bound": "fp64", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                       "frac": achieved / peak64, "flop_per_particle": taylor_flop_per_particle(p),
                       "peak_basis": "measured: the probe's fma.rn.f64 rate, this run"}
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
                    "pipe; in FP64 mode FP64 kernels (this library's mixed-radix transforms); Ewald-summed periodic "
                    "force = near + far"}


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
        # per step the forward needs only the positions and the adjoint also g, and the
        # accelerations can leave while the adjoint runs: the positions go up first, g
        # second; acc comes down after the forward, the gradient after the adjoint
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pos_in, g_in = [ev(), ev()], [ev(), ev()]
        fwd_done, comp_done, out_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]

        def upload(b):
            dpos[b].copy_(hp, non_blocking=True)
            pos_in[b].record(cin)
            dg[b].copy_(hg, non_blocking=True)
            g_in[b].record(cin)

        t0.record(stream)
        cin.wait_event(t0)
        with torch.cuda.stream(cin):
            upload(0)
        for i in range(n):
            b = i % 2
            if i + 1 < n:  # next step's upload into the other buffers, once step i-1 is done with them
                with torch.cuda.stream(cin):
                    if i >= 1:
                        cin.wait_event(comp_done[1 - b])
                    upload(1 - b)
            stream.wait_event(pos_in[b])
            if i >= 2:
                stream.wait_event(out_done[b])  # step i-2's download of these outputs
            flush.zero_()
            nf.forces(dpos[b], w.box, w.K, w.R, w.eps, out=dacc[b])
            fwd_done[b].record(stream)
            stream.wait_event(g_in[b])
            nf.forces_adjoint(dpos[b], dg[b], w.box, w.K, w.R, w.eps, out=dgr[b])
            comp_done[b].record(stream)
            with torch.cuda.stream(cout):
                cout.wait_event(fwd_done[b])
                ha.copy_(dacc[b], non_blocking=True)
                cout.wait_event(comp_done[b])
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
    # the pipelined run is as long as half the timed steps: only its first upload and last
    # download stand outside the compute, so a longer run is closer to a simulation's steady state
    n_pipe = max(3, args.steps // 2)
    t_pipe = pipelined(n_pipe)
    return {"value": 2 * P * n_pipe / t_pipe, "unit": UNIT, "h2d_bytes_per_step": 2 * w.pos.nbytes,
            "d2h_bytes_per_step": 2 * w.pos.nbytes, "steps": n_pipe, "serial_steps": n,
            "serial_value": 2 * P * n / tot,
            "note": "pinned host pos and g in, acc and grad out, every step; uploads and downloads on "
                    "their own streams overlapping the compute (positions first, g during the forward; "
                    "acc during the adjoint, the gradient after it; serial_value: one step at a time)"}


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
    # the autotuner picks the tuning of the batched launch on these boxes (measured afresh, no cache)
    run = nf.BatchedNearField(w.boxes, device=dev, tune="auto", tune_cache=None)
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

    # the same batch as a graph with the library's default tuning, for comparison
    base = nf.BatchedNearField(w.boxes, device=dev)
    base.pos.copy_(run.pos)
    base.capture()
    t_graph_default = timed(lambda: base())
    del base
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
            "separate_ms": t_sep * 1e3, "graph_default_tuning_ms": t_graph_default * 1e3,
            "tuning": {"picked": list(run.tune), "by": "autotune.tune on this batch (sinks per lane, stage, "
                       "warps per block, blocks per SM)", "candidates_ms": run.tune_timings,
                       "default": list(_lib.nf_get_default_tuning())}}


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
    g64 = g_np.astype(np.float64)
    t0 = time.perf_counter()
    grid = oracle.Grid(w.pos, w.box, w.K, w.R, w.eps)
    setup_s = time.perf_counter() - t0
    off, perm = grid.binning()
    counts = np.diff(off)
    S = stencil_sums(counts.reshape(w.K, w.K, w.K), w.R).reshape(-1)
    cost = counts.astype(np.int64) * S
    budget = max(2.0, 150.0 / (args.steps + args.warmup))
    C = w.K ** 3
    rate = None  # pairs/s of forces + adjoint, from the first step
    n_cells = max(1, C // 10000)
    times, pairs, sizes = [], [], []
    for k in range(args.warmup + args.steps):
        rng = np.random.default_rng(23 + k)
        cells = np.sort(rng.choice(C, n_cells, replace=False))
        mask = np.zeros(C, bool)
        mask[cells] = True
        sk = perm[np.repeat(mask, counts)].astype(np.int64)  # cell by cell
        t0 = time.perf_counter()
        grid.forces(sk)
        grid.adjoint(g64, sk)
        dt = time.perf_counter() - t0
        p = 2 * int(cost[cells].sum())
        if rate is None:
            # size every later sample to about `budget` seconds
            rate = p / max(dt, 1e-6)
            mean_cost = 2 * float(cost.mean())
            n_cells = int(min(C, max(1, budget * rate / max(mean_cost, 1.0))))
        if k >= args.warmup:
            times.append(dt)
            pairs.append(p)
            sizes.append(len(sk))
    grid.close()
    value = sum(pairs) / sum(times)
    sample = (f"forces + adjoint of every particle in {n_cells} random sink cells of {C} per step (fresh cells "
              f"each step, about {int(np.mean(sizes))} particles, listed cell by cell), FP64; the particle set binned once before "
              f"the steps ({setup_s:.1f} s, not timed per step)")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": describe(w), "step": "oracle forces + adjoint on a random sample of sink cells"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
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
