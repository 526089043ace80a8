"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle

# Parity bar for FP32 accelerations against the FP64 oracle (fractional error
# |a - a_ref| / |a_ref| per particle, no floor): median and maximum.
FORCE_MEDIAN = 1e-6
FORCE_MAX = 1e-4


def torch_cuda():
    import torch
    return torch


def to_dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def gpu_forces(w, tune=None, net=False):
    """Forces of a Workload through the C ABI (nf_forces or the batched entry)."""
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    torch = torch_cuda()
    pos = to_dev(w.pos)
    if tune is None:
        acc, nt = nf.forces(pos, w.box, w.K, w.R, w.eps, net=True)
    else:
        box = dict(N=w.N, K=w.K, R=w.R, eps=w.eps, box=w.box)
        arr = _lib.make_boxes([box])
        ws = torch.empty(_lib.nf_workspace_bytes_batched([box]), dtype=torch.uint8, device="cuda")
        acc = torch.empty_like(pos)
        nt = torch.empty((1, 3), dtype=torch.float64, device="cuda")
        _lib.nf_forces_batched(arr, pos, acc, nt, tune, ws)
        nt = nt[0]
    torch.cuda.synchronize()
    out = acc.cpu().numpy()
    return (out, nt.cpu().numpy()) if net else out


def frac_stats(a, ref):
    e = oracle.frac_error(a, ref)
    return float(np.median(e)), float(np.percentile(e, 99)), float(e.max())


def assert_force_parity(a, ref, median=FORCE_MEDIAN, maxerr=FORCE_MAX, label=""):
    assert np.all(np.isfinite(a)), f"{label}: non-finite output"
    med, p99, mx = frac_stats(a, ref)
    assert med <= median and mx <= maxerr, f"{label}: median {med:.3e} p99 {p99:.3e} max {mx:.3e}"
    return med, p99, mx


def sample_sinks(w, count, seed, include_densest=True):
    """Sampled sink indices: `count` random particles plus every particle of the
    densest cell (where FP32 accumulation is hardest)."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(w.N, size=min(count, w.N), replace=False)
    if include_densest:
        cid = oracle.cell_of(w.pos, w.box, w.K)
        dense = np.bincount(cid).argmax()
        idx = np.union1d(idx, np.nonzero(cid == dense)[0])
    return np.sort(idx)


def dense_pencil_with_close_pairs(seed: int = 21, K: int = 6, per_cell: int = 300, pairs: int = 20):
    """Positions (box 1) for the pair kernel's stage paths: a dense x-pencil of cells (j, k) = (2, 3),
    with `per_cell` particles in each cell (so a 128-sink chunk can lie inside one cell, away from the
    centre cell of its item or two cells from the source plane), plus close pairs (6e-4 box apart)
    straddling every x-face of the pencil and the y-face to its neighbour pencil.  With eps = 0.002
    (eps_s = 0.00432) the straddling pairs are inside the softening, so the stages holding them must
    take the exact path even where no self pair is present."""
    rng = np.random.default_rng(seed)
    w = 1.0 / K
    parts = []
    for i in range(K):
        parts.append((np.array([i, 2, 3]) + 0.5 + rng.uniform(-0.45, 0.45, (per_cell, 3))) * w)
    for i in range(K):
        xf = ((i + 1) % K) * w
        for _ in range(pairs):
            y, z = (2 + rng.uniform(0.05, 0.95)) * w, (3 + rng.uniform(0.05, 0.95)) * w
            parts.append(np.array([[xf - 3e-4, y, z], [xf + 3e-4, y + 1e-4, z]]))
        yf = 3 * w
        for _ in range(pairs):
            x, z = (i + rng.uniform(0.05, 0.95)) * w, (3 + rng.uniform(0.05, 0.95)) * w
            parts.append(np.array([[x, yf - 3e-4, z], [x + 1e-4, yf + 3e-4, z]]))
    x = np.concatenate(parts) % 1.0
    return x.astype(np.float32)
