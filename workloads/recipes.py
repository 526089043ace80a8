"""Seeded synthetic particle recipes.

The paper's own hot-path workload (a 512^3 LCDM snapshot, Sec. "Force
Accuracy", LCDM subsection) and its Ewald reference set are not available, so
these recipes stand in for them.  They keep the paper's structural choices:
about 64 particles per cell (Sec. "Two-Stage Execution": 30-100 per cell), a
softening of 1/40 of the mean interparticle spacing (Sec. "Outputs"), and
near-field radius R = 2 (5^3 neighbour cells, Sec. "GPU Near-Field
Computation").

Every draw uses ``numpy.random.Generator(PCG64(seed))`` in FP64.  Positions are
wrapped into the unit box, cast to FP32, and any value that rounds up to 1.0f
is mapped to 0.0f, so every coordinate lies in [0, 1).

Clustered recipe (order of draws is part of the definition):
  1. n_bg = round(0.4 N) background positions, uniform in the box.
  2. n_sph sphere masses M_k = 20 U^(-1/0.9) (a Pareto law with dN/dM ~ M^-1.9
     above 20).  Member counts are 20 + floor(s (M_k - 20)) with
     s = (n_cl - 20 n_sph) / sum(M_k - 20); the leftover particles go one by
     one to the spheres with the largest fractional parts, so the total is
     exact and every sphere keeps at least 20 members.
  3. n_sph sphere centres, uniform in the box.
  4. Per member: a Plummer radius r = a / sqrt(U^(-2/3) - 1) (inverse CDF of
     the Plummer mass profile) with scale radius a = 0.3 w (count/64)^(1/3),
     w the cell width; then an isotropic direction from a normalised
     3-D standard normal draw.  Positions are wrapped periodically.
  5. The whole set is shuffled by one permutation draw.

Nothing here computes forces, cells or offsets: it only draws inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _to_unit_f32(x: np.ndarray, box: float = 1.0) -> np.ndarray:
    """Wrap FP64 coordinates into [0, box), cast to FP32, map box -> 0."""
    y = np.mod(x, box).astype(np.float32)
    y[y >= np.float32(box)] = np.float32(0.0)
    return np.ascontiguousarray(y)


def plummer_eps(N: int, box: float = 1.0) -> float:
    """Plummer-equivalent softening: 1/40 of the mean interparticle spacing box/N^(1/3)."""
    r = round(N ** (1.0 / 3.0))
    cube_root = float(r) if r ** 3 == N else N ** (1.0 / 3.0)
    return box / (40.0 * cube_root)


def uniform_positions(N: int, seed: int, box: float = 1.0) -> np.ndarray:
    """N positions i.i.d. uniform in [0, box)^3, FP32 [N, 3]."""
    rng = _rng(seed)
    return _to_unit_f32(rng.random((N, 3)) * box, box)


def sphere_counts(n_cl: int, n_sph: int, rng: np.random.Generator) -> np.ndarray:
    """Member counts of the clustered recipe, step 2 (exact total, min 20)."""
    U = rng.random(n_sph)
    M = 20.0 * (1.0 - U) ** (-1.0 / 0.9)
    excess = M - 20.0
    s = (n_cl - 20 * n_sph) / excess.sum()
    raw = s * excess
    base = np.floor(raw)
    counts = (20 + base).astype(np.int64)
    left = int(n_cl - counts.sum())
    frac = raw - base
    order = np.argsort(-frac, kind="stable")
    counts[order[:left]] += 1
    assert counts.sum() == n_cl and counts.min() >= 20
    return counts


def clustered_positions(N: int, K: int, seed: int, n_sph: Optional[int] = None,
                        box: float = 1.0) -> np.ndarray:
    """Clustered recipe (see module docstring), FP32 [N, 3] in [0, box)."""
    rng = _rng(seed)
    n_bg = int(round(0.4 * N))
    n_cl = N - n_bg
    if n_sph is None:
        n_sph = max(1, N // 512)
    n_sph = max(1, min(n_sph, n_cl // 20))
    bg = rng.random((n_bg, 3)) * box
    if n_cl >= 20:
        counts = sphere_counts(n_cl, n_sph, rng)
        centres = rng.random((n_sph, 3)) * box
        w = box / K
        a = 0.3 * w * (counts / 64.0) ** (1.0 / 3.0)
        a_rep = np.repeat(a, counts)
        c_rep = np.repeat(centres, counts, axis=0)
        U = rng.random(n_cl)
        with np.errstate(divide="ignore"):
            r = a_rep / np.sqrt(U ** (-2.0 / 3.0) - 1.0)
        v = rng.standard_normal((n_cl, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        cl = c_rep + r[:, None] * v
    else:
        cl = rng.random((n_cl, 3)) * box
    x = np.concatenate([bg, cl], axis=0)
    x = x[rng.permutation(N)]
    return _to_unit_f32(x, box)


@dataclass
class Workload:
    """One or several periodic boxes of particles with their near-field parameters.

    eps is the Plummer-equivalent softening (box units); the method converts it
    internally.  For a batched workload, ``boxes`` lists per-box dicts with keys
    N, K, R, eps, box and the positions are concatenated in box order.
    """
    name: str
    pos: np.ndarray                 # FP32 [N_total, 3]
    box: float
    K: int
    R: int
    eps: float
    boxes: List[dict] = field(default_factory=list)

    @property
    def N(self) -> int:
        return int(self.pos.shape[0])


def config_plain(N: int = 32768, K: int = 8, seed: int = 0) -> Workload:
    """Plain forward: uniform positions, ~64 per cell, R = 2."""
    return Workload("plain", uniform_positions(N, seed), 1.0, K, 2, plummer_eps(N))


def config_clustered(N: int = 128 ** 3, K: int = 32, seed: int = 1,
                     n_sph: Optional[int] = None) -> Workload:
    """Clustered forward: 40 % uniform, 60 % in Plummer spheres."""
    if n_sph is None:
        n_sph = max(1, N // 512)
    return Workload("clustered", clustered_positions(N, K, seed, n_sph), 1.0, K, 2,
                    plummer_eps(N))


def config_large(N: int = 512 ** 3, K: int = 128, seed: int = 2) -> Workload:
    """Large forward: the clustered recipe scaled (N/512 spheres)."""
    return Workload("large", clustered_positions(N, K, seed, N // 512), 1.0, K, 2,
                    plummer_eps(N))


def config_adjoint(N: int = 64 ** 3, K: int = 16, seed: int = 3) -> Workload:
    """Adjoint: clustered recipe, loss L = sum_i g_i . a_i."""
    return Workload("adjoint", clustered_positions(N, K, seed, N // 512), 1.0, K, 2,
                    plummer_eps(N))


def upstream_gradient(N: int, seed: int = 33) -> np.ndarray:
    """g_i i.i.d. N(0, 1), FP32 [N, 3]."""
    return np.ascontiguousarray(_rng(seed).standard_normal((N, 3)).astype(np.float32))


def fd_sample(pos: np.ndarray, K: int, count: int = 256, seed: int = 333,
              min_face: float = 1e-5, box: float = 1.0) -> np.ndarray:
    """Indices of `count` particles at least `min_face` (box units) from every cell face.

    Finite differences move a particle by a small step; one that crosses a cell
    face changes its neighbour set, so such particles are excluded from the sample.
    """
    t = pos.astype(np.float64) * (K / box)
    gap = np.abs(t - np.round(t)).min(axis=1) * (box / K)
    ok = np.nonzero(gap >= min_face)[0]
    rng = _rng(seed)
    return np.sort(rng.choice(ok, size=min(count, ok.size), replace=False))


def config_batched(nboxes: int = 64, seed: int = 4, n_lo: int = 16 ** 3,
                   n_hi: int = 96 ** 3) -> Workload:
    """Batched: nboxes independent boxes, N_b log-uniform in [n_lo, n_hi].

    Box b uses the clustered recipe with seed 1000 + b, K_b = max(5, round((N_b/64)^(1/3))),
    eps_b = 1/(40 N_b^(1/3)) and round(N_b / 512) spheres.
    """
    rng = _rng(seed)
    lnN = rng.uniform(math.log(n_lo), math.log(n_hi), size=nboxes)
    boxes, parts = [], []
    for b in range(nboxes):
        Nb = int(round(math.exp(lnN[b])))
        Kb = max(5, int(round((Nb / 64.0) ** (1.0 / 3.0))))
        epsb = 1.0 / (40.0 * Nb ** (1.0 / 3.0))
        nsph = max(1, int(round(Nb / 512.0)))
        parts.append(clustered_positions(Nb, Kb, 1000 + b, nsph))
        boxes.append(dict(N=Nb, K=Kb, R=2, eps=epsb, box=1.0))
    pos = np.ascontiguousarray(np.concatenate(parts, axis=0))
    return Workload("batched", pos, 1.0, 0, 2, 0.0, boxes)


def named_config(name: str) -> Workload:
    return {
        "plain": config_plain,
        "clustered": config_clustered,
        "large": config_large,
        "adjoint": config_adjoint,
        "batched": config_batched,
    }[name]()
