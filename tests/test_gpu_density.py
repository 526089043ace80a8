"""nf_forces_density: the top-hat density estimate fused in the force kernel,
against the FP64 oracle; the accelerations stay bit-identical to nf_forces."""
import numpy as np
import pytest

import oracle
from workloads import config_clustered, config_plain
from workloads.recipes import Workload

from _helpers import sample_sinks, to_dev

pytestmark = pytest.mark.gpu

# Each term b^2 - r^2 is formed in FP32 from r^2 with a relative error of a
# few 1e-7 (cell-relative FP32 coordinates) and the terms are summed in FP32
# per stage, like the forces; rho >= 1 (the particle itself).  The bar is on
# the relative error |rho - rho_ref| / rho_ref: median and maximum.
RHO_MEDIAN = 1e-6
RHO_MAX = 1e-4


def _gpu(w, b):
    import torch
    import paper_2110_11392_gb300 as nf
    pos = to_dev(w.pos)
    acc, rho = nf.forces_density(pos, w.box, w.K, w.R, w.eps, b)
    plain = nf.forces(pos, w.box, w.K, w.R, w.eps)
    torch.cuda.synchronize()
    assert torch.equal(acc, plain), "accelerations must not change when the density is added"
    return rho.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("b_cells", [0.1, 0.5, 2.0])
def test_density_plain_full(b_cells):
    w = config_plain()
    b = b_cells * w.box / w.K
    rho = _gpu(w, b)
    ref = oracle.density(w.pos, w.box, w.K, w.R, b)
    err = np.abs(rho - ref) / ref
    assert np.median(err) <= RHO_MEDIAN and err.max() <= RHO_MAX, (np.median(err), err.max())
    assert rho.min() >= 1.0 - 1e-6


def test_density_clustered_sampled():
    w = config_clustered()
    b = 0.25 * w.box / w.K
    rho = _gpu(w, b)
    idx = sample_sinks(w, 5000, seed=7)
    ref = oracle.density(w.pos, w.box, w.K, w.R, b, sinks=idx)
    err = np.abs(rho[idx] - ref) / ref
    assert np.median(err) <= RHO_MEDIAN and err.max() <= RHO_MAX, (np.median(err), err.max())


def test_density_lattice_closed_form():
    K = 8
    g = np.arange(K) + 0.5
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    w = Workload("lattice", x, float(K), K, 2, 0.1)
    rho = _gpu(w, 1.5)
    assert np.allclose(rho, 17.0 / 3.0, rtol=0, atol=2e-6)


def test_density_radius_outside_near_field_is_rejected():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w = config_plain(N=4096, K=5)
    with pytest.raises(_lib.NFError):
        nf.forces_density(to_dev(w.pos), w.box, w.K, w.R, w.eps, 2.01 / w.K)
    torch.cuda.synchronize()


@pytest.mark.parametrize("b_cells", [0.05, 0.25, 0.5, 2.0])
def test_fused_and_deferred_density_are_bit_identical(b_cells):
    """The deferred top hat (a second sweep only over stages with a pair
    closer than b) runs the fused term's operations in the same order, so
    rho and acc must be equal bit for bit in both modes (and in auto)."""
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w = config_clustered(N=1 << 18, K=16)
    pos = to_dev(w.pos)
    b = b_cells * w.box / w.K
    before = _lib.nf_get_density_mode()
    out = {}
    try:
        for mode in (_lib.NF_DENS_FUSED, _lib.NF_DENS_DEFERRED, _lib.NF_DENS_AUTO):
            _lib.nf_set_density_mode(mode)
            out[mode] = nf.forces_density(pos, w.box, w.K, w.R, w.eps, b)
        torch.cuda.synchronize()
    finally:
        _lib.nf_set_density_mode(before)
    (a1, r1), (a2, r2), (a0, r0) = out[1], out[2], out[0]
    assert torch.equal(a1, a2) and torch.equal(a1, a0)
    assert torch.equal(r1, r2) and torch.equal(r1, r0)
    if b_cells <= 0.25:
        idx = sample_sinks(w, 2000, seed=11)
        ref = oracle.density(w.pos, w.box, w.K, w.R, b, sinks=idx)
        err = np.abs(r2.cpu().numpy().astype(np.float64)[idx] - ref) / ref
        assert np.median(err) <= RHO_MEDIAN and err.max() <= RHO_MAX, (np.median(err), err.max())
