"""nf_multipoles: complete-basis cell multipoles (Eq. multipoles) in FP64 on the
device, against the FP64 oracle's nested loops."""
import numpy as np
import pytest

import oracle
from workloads import config_adjoint, config_plain, uniform_positions

pytestmark = pytest.mark.gpu


def _gpu(pos, box, K, p):
    import torch
    import paper_2110_11392_gb300 as nf
    M = nf.multipoles(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), box, K, p)
    torch.cuda.synchronize()
    return M.cpu().numpy()


@pytest.mark.parametrize("p", [0, 1, 8, 16])
def test_multipoles_plain(p):
    w = config_plain()
    M = _gpu(w.pos, w.box, w.K, p)
    ref = oracle.multipoles(w.pos, w.box, w.K, p)
    assert M.shape == ref.shape
    tol = 1e-12 * np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    assert np.all(np.abs(M - ref) <= np.maximum(tol, 1e-13 * np.abs(ref)))


def test_multipoles_clustered_order8():
    w = config_adjoint()
    M = _gpu(w.pos, w.box, w.K, 8)
    ref = oracle.multipoles(w.pos, w.box, w.K, 8)
    rel = np.abs(M - ref) / (np.abs(ref) + 1e-12 * np.abs(ref).max(axis=0, keepdims=True) + 1e-300)
    assert rel.max() <= 1e-10
    # the monopole is the occupancy, exactly
    off, _, _ = oracle.bin_particles(w.pos, w.box, w.K)
    assert np.array_equal(M[:, 0], np.diff(off).astype(np.float64))


def test_multipoles_empty_cells_and_non_unit_box():
    x = uniform_positions(3000, 17, 2.0) * np.float32(0.5)   # half the box empty
    M = _gpu(x, 2.0, 6, 4)
    ref = oracle.multipoles(x, 2.0, 6, 4)
    assert np.allclose(M, ref, rtol=1e-12, atol=1e-15)
    assert np.count_nonzero(np.abs(M).sum(axis=1) == 0) > 0
