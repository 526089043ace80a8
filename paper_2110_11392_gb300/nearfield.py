"""PyTorch-facing API: workspaces, the autograd Function, and the batched graph runner.

PyTorch provides device memory and streams only.  Every step of the near-field
path (binning, work list, pair sums, adjoint, combine) runs in libnf's CUDA
kernels through the C ABI in :mod:`._lib`.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import _lib

_WS_CACHE = {}


def workspace(nbytes: int, device=None, key: str = "default") -> torch.Tensor:
    """A cached device workspace of at least nbytes (grown on demand, 256-byte aligned)."""
    device = torch.device(device if device is not None else "cuda")
    if device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    k = (device, key)
    buf = _WS_CACHE.get(k)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _WS_CACHE[k] = buf
    assert buf.data_ptr() % 256 == 0
    return buf


def _check_pos(pos: torch.Tensor) -> torch.Tensor:
    if not pos.is_cuda:
        raise ValueError("positions must be a CUDA tensor")
    if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError("positions must be float32 [N, 3]")
    return pos.contiguous()


def bin_particles(pos: torch.Tensor, box: float, K: int, ws: Optional[torch.Tensor] = None
                  ) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Stable binning (nf_bin): (cell_offsets int32[K^3+1], rel float32[N,4], perm int32[N])."""
    pos = _check_pos(pos)
    N = pos.shape[0]
    dev = pos.device
    off = torch.empty(K ** 3 + 1, dtype=torch.int32, device=dev)
    rel = torch.empty((N, 4), dtype=torch.float32, device=dev)
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(_lib.nf_workspace_bytes(N, max(K, 5), 2), dev)
    _lib.nf_bin(pos, box, K, off, rel, perm, ws)
    return off, rel, perm


def forces(pos: torch.Tensor, box: float, K: int, R: int, eps: float,
           ws: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
           net: bool = False):
    """Near-field accelerations (nf_forces), float32 [N, 3] in input order.

    eps is the Plummer-equivalent softening (box units).  With net=True also
    returns the FP64 sum of m a (a float64 [3] tensor).
    """
    pos = _check_pos(pos)
    N = pos.shape[0]
    if ws is None:
        ws = workspace(_lib.nf_workspace_bytes(N, K, R), pos.device)
    acc = out if out is not None else torch.empty_like(pos)
    net_t = torch.empty(3, dtype=torch.float64, device=pos.device) if net else None
    _lib.nf_forces(pos, box, K, R, eps, acc, net_t, ws)
    return (acc, net_t) if net else acc


def forces_density(pos: torch.Tensor, box: float, K: int, R: int, eps: float, b: float,
                   ws: Optional[torch.Tensor] = None):
    """Accelerations and the top-hat density estimate (nf_forces_density):
    (acc float32 [N, 3], rho float32 [N]), rho_i = sum_{r_ij < b} (1 - r_ij^2/b^2)."""
    pos = _check_pos(pos)
    N = pos.shape[0]
    if ws is None:
        ws = workspace(_lib.nf_workspace_bytes(N, K, R), pos.device)
    acc = torch.empty_like(pos)
    rho = torch.empty(N, dtype=torch.float32, device=pos.device)
    _lib.nf_forces_density(pos, box, K, R, eps, b, acc, rho, ws)
    return acc, rho


def forces_adjoint(pos: torch.Tensor, g: torch.Tensor, box: float, K: int, R: int, eps: float,
                   ws: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None):
    """dL/dx for upstream g = dL/da (nf_forces_adjoint), float32 [N, 3]."""
    pos = _check_pos(pos)
    g = g.to(torch.float32).contiguous()
    if g.shape != pos.shape:
        raise ValueError("g must have the shape of pos")
    N = pos.shape[0]
    if ws is None:
        ws = workspace(_lib.nf_workspace_bytes(N, K, R), pos.device)
    grad = out if out is not None else torch.empty_like(pos)
    _lib.nf_forces_adjoint(pos, g, box, K, R, eps, grad, ws)
    return grad


def multipoles(pos: torch.Tensor, box: float, K: int, p: int, ws: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Complete-basis cell multipoles (nf_multipoles): float64 [K^3, (p+3)(p+2)(p+1)/6]."""
    pos = _check_pos(pos)
    N = pos.shape[0]
    if ws is None:
        ws = workspace(_lib.nf_workspace_bytes(N, max(K, 5), 2), pos.device)
    M = torch.empty((K ** 3, (p + 3) * (p + 2) * (p + 1) // 6), dtype=torch.float64, device=pos.device)
    _lib.nf_multipoles(pos, box, K, p, M, ws)
    return M


class FarField:
    """The far field of one grid (nf_derivatives once, nf_far_forces per call).

    f = FarField(K, R, p, box); a_far = f(pos); or f(pos, add_to=acc) adds the
    far acceleration into an FP32 [N, 3] tensor (e.g. the output of forces()).
    """

    def __init__(self, K: int, R: int, p: int, box: float = 1.0, device=None):
        self.K, self.R, self.p, self.box = int(K), int(R), int(p), float(box)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = _lib.nf_derivatives_bytes(self.K, self.p)
        if nbytes == 0:
            raise ValueError(f"far field: K = {K}, p = {p} out of range")
        self.derivs = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        ws = torch.empty(_lib.nf_far_workspace_bytes(1, self.K, self.p), dtype=torch.uint8, device=self.device)
        _lib.nf_derivatives(self.K, self.R, self.p, self.box, self.derivs, ws)
        self.nterms = (self.p + 3) * (self.p + 2) * (self.p + 1) // 6

    def workspace(self, N: int) -> torch.Tensor:
        return workspace(_lib.nf_far_workspace_bytes(N, self.K, self.p), self.device, key="far")

    def total(self, pos: torch.Tensor, eps: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The periodic force near + far (nf_forces_total), FP32 [N, 3]: one binning for both."""
        pos = _check_pos(pos)
        N = pos.shape[0]
        acc = out if out is not None else torch.empty_like(pos)
        ws = workspace(_lib.nf_workspace_bytes(N, self.K, self.R), self.device)
        _lib.nf_forces_total(pos, self.box, self.K, self.R, eps, self.p, self.derivs, acc, ws, self.workspace(N))
        return acc

    def __call__(self, pos: torch.Tensor, add_to: Optional[torch.Tensor] = None, want_far: bool = True,
                 want_taylors: bool = False, ws: Optional[torch.Tensor] = None):
        pos = _check_pos(pos)
        N = pos.shape[0]
        if ws is None:
            ws = self.workspace(N)
        acc = torch.empty((N, 3), dtype=torch.float64, device=pos.device) if want_far else None
        T = (torch.empty((self.K ** 3, self.nterms), dtype=torch.float64, device=pos.device)
             if want_taylors else None)
        _lib.nf_far_forces(pos, self.box, self.K, self.R, self.p, self.derivs, acc, add_to, T, ws)
        if want_taylors:
            return acc, T
        return acc


def status(ws: Optional[torch.Tensor] = None, N: int = 1, K: int = 5, R: int = 2) -> int:
    """Device status of the last call on the default workspace (synchronises)."""
    if ws is None:
        ws = workspace(0)
    return _lib.nf_status_read(ws)


def stats(ws: Optional[torch.Tensor] = None) -> dict:
    if ws is None:
        ws = workspace(0)
    return _lib.nf_stats_read(ws)


class NearField(torch.autograd.Function):
    """a = NearField.apply(pos, box, K, R, eps); backward runs the hand-written adjoint kernel.

    Only pos is saved; the backward pass recomputes the binning and the pair
    quantities (nothing per pair is stored).
    """

    @staticmethod
    def forward(ctx, pos, box, K, R, eps):
        ctx.save_for_backward(pos)
        ctx.params = (float(box), int(K), int(R), float(eps))
        return forces(pos, box, K, R, eps)

    @staticmethod
    def backward(ctx, g):
        (pos,) = ctx.saved_tensors
        box, K, R, eps = ctx.params
        grad = forces_adjoint(pos.detach(), g, box, K, R, eps)
        return grad, None, None, None, None


def near_field(pos: torch.Tensor, box: float, K: int, R: int, eps: float) -> torch.Tensor:
    return NearField.apply(pos, box, K, R, eps)


class BatchedNearField:
    """Many independent boxes in one pass (nf_forces_batched), optionally as a CUDA graph.

    boxes: list of dicts with N, K, R, eps, box (packed back to back in pos_cat).
    tune: (sinks_per_lane, stage, warps_per_block, blocks_per_sm), None for the
    library default, or "auto": the autotuner (autotune.tune, cached in
    tune_cache; None = always measure) picks the tuning on the first call's
    positions, before any graph capture; the pick is in .tune and the
    candidates' times in .tune_timings.
    """

    def __init__(self, boxes: Sequence[dict], device=None, tune=None, net: bool = False,
                 tune_cache: Optional[str] = "default"):
        self.device = torch.device(device if device is not None else "cuda")
        self.boxes = [dict(b) for b in boxes]
        self.arr = _lib.make_boxes(self.boxes)
        self.N = sum(int(b["N"]) for b in self.boxes)
        self._auto = isinstance(tune, str) and tune == "auto"
        if isinstance(tune, str) and not self._auto:
            raise ValueError(f"tune must be a tuple, None or 'auto', not {tune!r}")
        self.tune = None if self._auto else tune
        self.tune_timings = None
        self.tune_cache = tune_cache
        nbytes = _lib.nf_workspace_bytes_batched(self.boxes)
        if nbytes == 0:
            raise ValueError("invalid batch: " + _lib.nf_last_error())
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.pos = torch.zeros((self.N, 3), dtype=torch.float32, device=self.device)
        self.acc = torch.zeros((self.N, 3), dtype=torch.float32, device=self.device)
        self.net = torch.zeros((len(self.boxes), 3), dtype=torch.float64, device=self.device) if net else None
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    def _launch(self):
        _lib.nf_forces_batched(self.arr, self.pos, self.acc, self.net, self.tune, self.ws)

    def _ensure_tuned(self):
        if self._auto and self.tune is None:
            from . import autotune
            cache = autotune.DEFAULT_CACHE if self.tune_cache == "default" else self.tune_cache
            self.tune, self.tune_timings = autotune.tune(self.boxes, self.pos, cache=cache)

    def __call__(self, pos_cat: Optional[torch.Tensor] = None) -> torch.Tensor:
        if pos_cat is not None:
            self.pos.copy_(pos_cat)
        if self.graph is not None:
            self.graph.replay()
        else:
            self._ensure_tuned()
            self._launch()
        return self.acc

    def capture(self) -> "BatchedNearField":
        """Record one batched call into a CUDA graph (replayed by __call__).
        With tune="auto" the search runs first, on the positions held now."""
        self._ensure_tuned()
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self._launch()  # warm-up outside capture (kernel attributes, module load)
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._launch()
        self.graph = g
        return self

    def stats(self) -> dict:
        return _lib.nf_stats_read(self.ws)

    def status(self) -> int:
        return _lib.nf_status_read(self.ws)
