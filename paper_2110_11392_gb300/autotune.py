"""Autotuner of the pair kernel's work shape (sinks per lane, stage size, warps per block,
blocks per SM).

Each candidate is timed on the caller's workload through ``nf_forces_batched``
(or its adjoint) with CUDA events on the current stream; the fastest one is
returned and cached in a JSON file keyed by GPU name, direction and a coarse
problem class (particles per box and boxes), so later runs reuse it.  A cached
record is used only when it was measured over the same candidate list.
``BatchedNearField(tune="auto")`` runs this search before its first launch.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import _lib

Tuning = Tuple[int, int, int, int]

CANDIDATES: List[Tuning] = [
    (2, 128, 8, 0), (2, 64, 8, 0), (2, 128, 4, 0), (3, 128, 8, 0), (3, 64, 8, 0), (4, 128, 8, 0), (4, 64, 8, 0),
    (2, 128, 8, 3), (2, 64, 8, 3), (1, 128, 8, 3), (1, 64, 8, 3), (1, 128, 8, 0),
    (4, 128, 8, 1), (3, 128, 8, 1),
]

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "nf_tuning.json")


def problem_class(boxes: Sequence[dict], adjoint: bool) -> str:
    n = sum(int(b["N"]) for b in boxes)
    occ = n / max(1, sum(int(b["K"]) ** 3 for b in boxes))
    return (f"{'adj' if adjoint else 'fwd'}:logN={int(math.log2(max(n, 1)))}:"
            f"boxes={min(len(boxes), 64)}:occ={int(round(occ / 16.0)) * 16}")


def _time(fn, reps: int) -> float:
    s = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune(boxes: Sequence[dict], pos: torch.Tensor, adjoint: bool = False, g: Optional[torch.Tensor] = None,
         candidates: Sequence[Tuning] = CANDIDATES, reps: int = 3, cache: Optional[str] = DEFAULT_CACHE,
         refresh: bool = False) -> Tuple[Tuning, Dict[str, float]]:
    """Best tuning for this batch (pos packed as in nf_forces_batched) and the timings (ms)."""
    dev = pos.device
    key = f"{torch.cuda.get_device_name(dev)}|{problem_class(boxes, adjoint)}"
    cand_list = [list(map(int, t)) for t in candidates]
    if cache and not refresh and os.path.exists(cache):
        try:
            rec = json.load(open(cache)).get(key)
            if rec and rec.get("candidates") == cand_list:
                return tuple(rec["best"]), rec["ms"]
        except (OSError, ValueError, AttributeError):
            pass
    arr = _lib.make_boxes(boxes)
    ws = torch.empty(_lib.nf_workspace_bytes_batched(boxes), dtype=torch.uint8, device=dev)
    out = torch.empty_like(pos)
    if adjoint and g is None:
        g = torch.ones_like(pos)
    timings: Dict[str, float] = {}
    for t in candidates:
        if adjoint:
            fn = lambda t=t: _lib.nf_forces_adjoint_batched(arr, pos, g, out, t, ws)  # noqa: E731
        else:
            fn = lambda t=t: _lib.nf_forces_batched(arr, pos, out, None, t, ws)  # noqa: E731
        timings[",".join(map(str, t))] = _time(fn, reps)
    best = min(timings, key=timings.get)
    best_t = tuple(int(x) for x in best.split(","))
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            data = json.load(open(cache)) if os.path.exists(cache) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = {"best": list(best_t), "ms": timings, "candidates": cand_list}
        try:
            with open(cache, "w") as fh:
                json.dump(data, fh, indent=1)
        except OSError:
            pass
    return best_t, timings


def tune_single(pos: torch.Tensor, box: float, K: int, R: int, eps: float, adjoint: bool = False,
                g: Optional[torch.Tensor] = None, **kw) -> Tuple[Tuning, Dict[str, float]]:
    boxes = [dict(N=pos.shape[0], K=K, R=R, eps=eps, box=box)]
    return tune(boxes, pos, adjoint=adjoint, g=g, **kw)
