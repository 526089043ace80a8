"""nf_forces on the GPU against the FP64 oracle (median <= 1e-6, max <= 1e-4)."""
import numpy as np
import pytest

import oracle
from workloads import clustered_positions, config_adjoint, config_clustered, config_plain, uniform_positions
from workloads.recipes import Workload

from _helpers import assert_force_parity, dense_pencil_with_close_pairs, gpu_forces, sample_sinks

pytestmark = pytest.mark.gpu


def test_plain_config_full_oracle():
    w = config_plain()
    acc, net = gpu_forces(w, net=True)
    ref = oracle.forces(w.pos, w.box, w.K, w.R, w.eps)
    assert_force_parity(acc, ref, label="plain")
    # Newton III: the FP64 sum of m a over FP32 results is at FP32 roundoff
    scale = np.abs(acc).sum() / w.N
    assert np.abs(net).max() <= 1e-6 * scale
    assert np.allclose(net, acc.astype(np.float64).sum(axis=0) / w.N, rtol=1e-9, atol=1e-12 * scale)


def test_adjoint_config_forward_full_oracle():
    w = config_adjoint()
    acc = gpu_forces(w)
    ref = oracle.forces(w.pos, w.box, w.K, w.R, w.eps)
    assert_force_parity(acc, ref, label="clustered 64^3")


def test_clustered_config_sampled_sinks():
    w = config_clustered()
    acc = gpu_forces(w)
    idx = sample_sinks(w, 6000, seed=101)
    ref = oracle.forces(w.pos, w.box, w.K, w.R, w.eps, sinks=idx)
    assert_force_parity(acc[idx], ref, label="clustered 128^3 sampled")


def test_tiny_box_matches_minimum_image_brute_force():
    """K = 5: the stencil is the whole box; jittered particles make the cell
    image the minimum image, so the GPU matches a textbook O(N^2) sum."""
    rng = np.random.default_rng(11)
    K, w_ = 5, 0.2
    cells = rng.integers(0, K, size=(3000, 3))
    x = ((cells + 0.5) * w_ + rng.uniform(-0.24 * w_, 0.24 * w_, size=(3000, 3))).astype(np.float32)
    eps = 0.002
    w = Workload("tiny", x, 1.0, K, 2, eps)
    acc = gpu_forces(w)
    xd = x.astype(np.float64)
    d = xd[None, :, :] - xd[:, None, :]
    d -= np.round(d)
    r = np.linalg.norm(d, axis=2)
    es = 2.16 * eps
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(r < es, (10 - 15 * r / es + 6 * (r / es) ** 2) / es ** 3, 1 / r ** 3)
    f[r == 0] = 0
    ref = (f[:, :, None] * d).sum(axis=1) / len(x)
    assert_force_parity(acc, ref, label="brute force")


def test_lattice_is_force_free():
    K = 8
    g = np.arange(K) + 0.5
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    w = Workload("lattice", x, float(K), K, 2, 0.1)
    acc = gpu_forces(w)
    # exact symmetry; FP32 sums of +-terms cancel to roundoff of m/w^2 = 1/N
    assert np.abs(acc).max() <= 1e-6 / len(x)


@pytest.mark.parametrize("N,K,R,box,seed", [
    (1, 5, 2, 1.0, 0),
    (2, 5, 2, 1.0, 1),
    (1000, 5, 1, 1.0, 2),
    (5000, 8, 3, 1.0, 3),
    (5000, 9, 4, 1.0, 4),
    (20000, 7, 2, 3.7, 5),
    (70001, 11, 2, 1.0, 6),
])
def test_ragged_sizes_and_radii(N, K, R, box, seed):
    x = uniform_positions(N, seed, box)
    eps = box / (40.0 * N ** (1 / 3)) if N > 8 else 0.01 * box
    w = Workload("ragged", x, box, K, R, eps)
    acc = gpu_forces(w)
    ref = oracle.forces(x, box, K, R, eps)
    if N == 1:
        assert np.array_equal(acc, np.zeros((1, 3), np.float32))
        return
    assert_force_parity(acc, ref, label=f"N={N} K={K} R={R}")


def test_one_cell_holds_everything():
    rng = np.random.default_rng(4)
    x = (0.5 + 0.01 * rng.standard_normal((3000, 3))).astype(np.float32)
    w = Workload("one-cell", x, 1.0, 5, 2, 1e-4)
    acc = gpu_forces(w)
    ref = oracle.forces(x, 1.0, 5, 2, 1e-4)
    assert_force_parity(acc, ref, label="one cell")


def test_softening_regime_and_coincident_particles():
    """Many pairs inside eps_s, exact duplicates (d = 0) and self pairs."""
    rng = np.random.default_rng(7)
    base = rng.random((400, 3)).astype(np.float32)
    near = (base + 0.002 * rng.standard_normal((400, 3))).astype(np.float32) % np.float32(1.0)
    x = np.concatenate([base, near, base[:50]])      # 50 exact duplicates
    eps = 0.004                                       # eps_s = 0.00864: many soft pairs
    w = Workload("soft", x, 1.0, 6, 2, eps)
    acc = gpu_forces(w)
    ref = oracle.forces(x, 1.0, 6, 2, eps)
    assert_force_parity(acc, ref, label="softened pairs")


@pytest.mark.parametrize("tune", [None, (4, 64, 8, 0), (2, 128, 8, 0), (1, 128, 4, 0), (4, 128, 8, 1)])
def test_dense_pencil_with_close_pairs_across_faces(tune):
    """Chunks inside one cell away from their item's centre cell run the centre cell's stages on
    the tracked fast path, chunks two cells from the source plane skip the tracking; the close
    pairs straddling the faces must still reach the exact (softened) branch."""
    x = dense_pencil_with_close_pairs()
    w = Workload("dense-pencil", x, 1.0, 6, 2, 0.002)
    acc = gpu_forces(w, tune=tune)
    ref = oracle.forces(x, 1.0, 6, 2, 0.002)
    assert_force_parity(acc, ref, label=f"dense pencil {tune}")


def test_empty_regions_and_clustered_voids():
    x = uniform_positions(30000, 11) * np.float32(0.5)
    w = Workload("half", x, 1.0, 16, 2, 1e-3)
    assert_force_parity(gpu_forces(w), oracle.forces(x, 1.0, 16, 2, 1e-3), label="half box")
    y = clustered_positions(100000, 12, 13, n_sph=10)
    w = Workload("voids", y, 1.0, 12, 2, 1e-3)
    idx = sample_sinks(w, 3000, seed=5)
    assert_force_parity(gpu_forces(w)[idx], oracle.forces(y, 1.0, 12, 2, 1e-3, sinks=idx), label="voids")


@pytest.mark.parametrize("tune", [(1, 64, 4, 0), (2, 128, 8, 0), (4, 64, 8, 0), (4, 128, 4, 1),
                                  (2, 64, 8, 2), (3, 128, 8, 1), (4, 128, 8, 1)])
def test_all_tunings_meet_parity(tune):
    w = config_plain()
    acc = gpu_forces(w, tune=tune)
    ref = oracle.forces(w.pos, w.box, w.K, w.R, w.eps)
    assert_force_parity(acc, ref, label=str(tune))


def test_deterministic():
    w = config_plain(N=50000, K=9, seed=8)
    a = gpu_forces(w)
    b = gpu_forces(w)
    assert np.array_equal(a, b)


def test_scaling_law_on_gpu():
    x = uniform_positions(20000, 21)
    a1 = gpu_forces(Workload("s1", x, 1.0, 8, 2, 1e-3))
    a2 = gpu_forces(Workload("s2", x * np.float32(2.0), 2.0, 8, 2, 2e-3))
    # cell-unit arithmetic is identical; only the final FP64 scale differs by 4
    assert np.array_equal(a1, a2 * np.float32(4.0))


def test_stats_pair_count():
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_plain()
    nf.forces(torch.from_numpy(w.pos).cuda(), w.box, w.K, w.R, w.eps)
    st = nf.stats()
    off, _, _ = oracle.bin_particles(w.pos, w.box, w.K)
    n = np.diff(off).reshape(w.K, w.K, w.K).astype(np.int64)
    S = np.zeros_like(n)
    for a in range(-2, 3):
        for b in range(-2, 3):
            for c in range(-2, 3):
                S += np.roll(n, (a, b, c), axis=(0, 1, 2))
    assert st["pairs"] == int((n * S).sum())
    assert st["max_occupancy"] == int(n.max())
    assert st["lane_pairs"] >= st["pairs"]


def test_stage_counters_match_the_work_list():
    """nf_stage_stats_read: the pair kernel's stages and exact-from-start stages equal the count
    implied by the cell occupancies (each pencil chunk runs its centre cell's sources in
    stages of their own, the rest of the plane in stages of the tuning's size; only the
    chunks holding sinks of the centre cell run those stages exactly from the start);
    re-runs are rare and never more than the fast stages."""
    import torch
    from paper_2110_11392_gb300 import _lib
    from workloads import config_adjoint
    w = config_adjoint()
    off, _, _ = oracle.bin_particles(w.pos, w.box, w.K)
    n = np.diff(off).reshape(w.K, w.K, w.K).astype(np.int64)
    R = w.R
    sink = sum(np.roll(n, -c, axis=0) for c in range(-R, R + 1))
    before = sum(np.roll(n, -c, axis=0) for c in range(-R, 0))    # sinks of the pencil ahead of its centre cell
    src = sum(np.roll(n, (-b, -d), axis=(1, 2)) for b in range(-R, R + 1) for d in range(-R, R + 1))
    pos = torch.from_numpy(w.pos).cuda()
    g = torch.from_numpy(np.ones_like(w.pos)).cuda()
    ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, R), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(pos)
    for adjoint, tune in ((False, _lib.nf_get_default_tuning()), (True, _lib.nf_get_default_tuning_adjoint())):
        S, B = tune[0], tune[1]
        CH = 32 * S
        nch = (sink + CH - 1) // CH
        self_chunks = np.where(n > 0, (before + n + CH - 1) // CH - before // CH, 0)
        assert (self_chunks <= nch).all()
        exact = int((self_chunks * ((n + B - 1) // B)).sum())
        total = int((nch * ((n + B - 1) // B + (src - n + B - 1) // B)).sum())
        if adjoint:
            _lib.nf_forces_adjoint(pos, g, w.box, w.K, R, w.eps, out, ws)
        else:
            _lib.nf_forces(pos, w.box, w.K, R, w.eps, out, None, ws)
        st = _lib.nf_stage_stats_read(ws)
        assert st["stages"] == total and st["exact"] == exact, (adjoint, st, total, exact)
        assert 0 <= st["rerun"] <= total - exact
