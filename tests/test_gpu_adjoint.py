"""nf_forces_adjoint and the autograd Function against the FP64 oracle gradient and
central finite differences of the local energy (cells frozen)."""
import numpy as np
import pytest

import oracle
from workloads import config_adjoint, config_plain, fd_sample, uniform_positions, upstream_gradient
from workloads.recipes import Workload

from _helpers import dense_pencil_with_close_pairs, frac_stats, to_dev

pytestmark = pytest.mark.gpu

# Gradient parity bar (fractional error per particle, FP32 kernel vs FP64 oracle).
# The adjoint sums J (g_j - g_i) with terms of either sign; it is held to the
# same bar as the forces.
ADJ_MEDIAN = 1e-6
ADJ_MAX = 1e-4


def _gpu_grad(w, g):
    import torch
    import paper_2110_11392_gb300 as nf
    pos = to_dev(w.pos)
    out = nf.forces_adjoint(pos, to_dev(g), w.box, w.K, w.R, w.eps)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_adjoint_plain_full_oracle():
    w = config_plain()
    g = upstream_gradient(w.N, 33)
    grad = _gpu_grad(w, g)
    ref = oracle.adjoint(w.pos, g.astype(np.float64), w.box, w.K, w.R, w.eps)
    med, p99, mx = frac_stats(grad, ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (med, p99, mx)


def test_adjoint_config_fd_and_oracle():
    """Clustered 64^3 box, 256 particles away from cell faces: the kernel's
    gradient agrees with the FP64 oracle gradient and with central finite
    differences (h = 1e-6 box) of the local energy."""
    w = config_adjoint()
    g = upstream_gradient(w.N, 33)
    grad = _gpu_grad(w, g)
    ks = fd_sample(w.pos, w.K, 256, 333)
    ref = oracle.adjoint(w.pos, g.astype(np.float64), w.box, w.K, w.R, w.eps, sinks=ks)
    med, p99, mx = frac_stats(grad[ks], ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (med, p99, mx)
    fd = oracle.fd_gradient(w.pos, g.astype(np.float64), w.box, w.K, w.R, w.eps, ks, h=1e-6)
    fmed, _, fmx = frac_stats(grad[ks], fd)
    # FD truncation (h^2 f''') and cancellation add their own error on top
    assert fmed <= 1e-5 and fmx <= 1e-2, (fmed, fmx)


def test_adjoint_config_sampled_full_gradient():
    w = config_adjoint()
    g = upstream_gradient(w.N, 33)
    grad = _gpu_grad(w, g)
    rng = np.random.default_rng(17)
    ks = np.sort(rng.choice(w.N, 4000, replace=False))
    ref = oracle.adjoint(w.pos, g.astype(np.float64), w.box, w.K, w.R, w.eps, sinks=ks)
    med, p99, mx = frac_stats(grad[ks], ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (med, p99, mx)


def test_autograd_function_runs_the_adjoint_kernel():
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_plain(N=20000, K=8, seed=5)
    g = upstream_gradient(w.N, 7)
    pos = to_dev(w.pos).requires_grad_(True)
    acc = nf.near_field(pos, w.box, w.K, w.R, w.eps)
    (acc * to_dev(g)).sum().backward()
    direct = nf.forces_adjoint(pos.detach(), to_dev(g), w.box, w.K, w.R, w.eps)
    assert torch.equal(pos.grad, direct)
    fwd = nf.forces(pos.detach(), w.box, w.K, w.R, w.eps)
    assert torch.equal(acc.detach(), fwd)


def test_adjoint_softened_and_coincident_pairs():
    rng = np.random.default_rng(7)
    base = rng.random((400, 3)).astype(np.float32)
    near = ((base + 0.002 * rng.standard_normal((400, 3))) % 1.0).astype(np.float32)
    x = np.concatenate([base, near, base[:50]])
    w = Workload("soft", x, 1.0, 6, 2, 0.004)
    g = rng.standard_normal(x.shape).astype(np.float32)
    grad = _gpu_grad(w, g)
    ref = oracle.adjoint(x, g.astype(np.float64), 1.0, 6, 2, 0.004)
    med, p99, mx = frac_stats(grad, ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (med, p99, mx)


def test_adjoint_dense_pencil_with_close_pairs_across_faces():
    """The adjoint's stage paths on dense single-cell chunks and close pairs across cell faces."""
    x = dense_pencil_with_close_pairs(seed=22)
    w = Workload("dense-pencil", x, 1.0, 6, 2, 0.002)
    g = np.random.default_rng(23).standard_normal(x.shape).astype(np.float32)
    grad = _gpu_grad(w, g)
    ref = oracle.adjoint(x, g.astype(np.float64), 1.0, 6, 2, 0.002)
    med, p99, mx = frac_stats(grad, ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (med, p99, mx)


@pytest.mark.parametrize("N,K,R", [(1, 5, 2), (3000, 5, 1), (9000, 9, 4)])
def test_adjoint_ragged(N, K, R):
    x = uniform_positions(N, 40 + N)
    g = upstream_gradient(N, 41)
    eps = 1.0 / (40.0 * max(N, 8) ** (1 / 3))
    w = Workload("ragged", x, 1.0, K, R, eps)
    grad = _gpu_grad(w, g)
    if N == 1:
        assert np.array_equal(grad, np.zeros((1, 3), np.float32))
        return
    ref = oracle.adjoint(x, g.astype(np.float64), 1.0, K, R, eps)
    med, p99, mx = frac_stats(grad, ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (med, p99, mx)


@pytest.mark.parametrize("tune", [(1, 64, 4, 0), (2, 128, 8, 0), (4, 128, 8, 0), (3, 128, 8, 1), (4, 128, 8, 1)])
def test_adjoint_tunings_meet_parity(tune):
    """The adjoint kernel variants (sinks per lane, stage, warps, blocks per SM; one block per SM
    selects the build with the whole register file) against the FP64 oracle gradient."""
    import torch
    from paper_2110_11392_gb300 import _lib
    w = config_plain()
    g = upstream_gradient(w.N, 34)
    box = dict(N=w.N, K=w.K, R=w.R, eps=w.eps, box=w.box)
    arr = _lib.make_boxes([box])
    ws = torch.empty(_lib.nf_workspace_bytes_batched([box]), dtype=torch.uint8, device="cuda")
    pos = to_dev(w.pos)
    out = torch.empty_like(pos)
    _lib.nf_forces_adjoint_batched(arr, pos, to_dev(g), out, tune, ws)
    torch.cuda.synchronize()
    ref = oracle.adjoint(w.pos, g.astype(np.float64), w.box, w.K, w.R, w.eps)
    med, p99, mx = frac_stats(out.cpu().numpy(), ref)
    assert med <= ADJ_MEDIAN and mx <= ADJ_MAX, (tune, med, p99, mx)
