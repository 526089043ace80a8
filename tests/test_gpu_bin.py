"""nf_bin on the GPU against the oracle: bit-exact cell offsets, permutation and offsets."""
import numpy as np
import pytest

import oracle
from workloads import clustered_positions, config_adjoint, config_clustered, config_plain, uniform_positions

pytestmark = pytest.mark.gpu


def _gpu_bin(pos, box, K):
    import torch
    import paper_2110_11392_gb300 as nf
    off, rel, perm = nf.bin_particles(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), box, K)
    torch.cuda.synchronize()
    return off.cpu().numpy(), rel.cpu().numpy(), perm.cpu().numpy()


def _assert_bit_exact(pos, box, K):
    off_g, rel_g, perm_g = _gpu_bin(pos, box, K)
    off_o, rel_o, perm_o = oracle.bin_particles(pos, box, K)
    assert np.array_equal(off_g, off_o), "cell offsets differ"
    assert np.array_equal(perm_g, perm_o), "permutation differs"
    assert np.array_equal(rel_g.view(np.int32), rel_o.view(np.int32)), "offset bits differ"


@pytest.mark.parametrize("name", ["plain", "adjoint", "clustered"])
def test_bin_configs_bit_exact(name):
    w = {"plain": config_plain, "adjoint": config_adjoint, "clustered": config_clustered}[name]()
    _assert_bit_exact(w.pos, w.box, w.K)


@pytest.mark.parametrize("N,K,box,seed", [
    (1, 5, 1.0, 0),
    (7, 5, 1.0, 1),
    (1000, 7, 3.7, 2),        # 9-bit keys: one sort pass, box != 1, K not a power of two
    (70001, 11, 1.0, 3),      # 11-bit keys: two passes; ragged last tile
    (300000, 24, 2.5, 4),     # 14-bit keys: two passes
    (1 << 20, 128, 1.0, 5),   # 21-bit keys: three 7-bit passes, 512 tiles
    (20000, 520, 1.0, 10),    # 28-bit keys: four passes, nearly every cell empty
    (200000, 24, 2.0, 6),     # K / box = 12: dyadic, integer shift path
    (200000, 10, 0.625, 7),   # K / box = 16
    (200000, 13, 1.3, 8),     # K / box = 10 (box not dyadic): FP64 shift path
])
def test_bin_uniform_sizes(N, K, box, seed):
    _assert_bit_exact(uniform_positions(N, seed, box), box, K)


def test_bin_adversarial_positions():
    K = 8
    one_minus = np.nextafter(np.float32(1.0), np.float32(0.0))
    rng = np.random.default_rng(9)
    faces = (rng.integers(0, K + 1, size=(2000, 3)) / K).astype(np.float32)   # exactly on faces, incl. 1.0
    edge = np.full((500, 3), one_minus, np.float32)
    dup = np.repeat(rng.random((10, 3)).astype(np.float32), 50, axis=0)        # duplicates keep order
    outside = (rng.random((500, 3)) * 5 - 2).astype(np.float32)               # wrapped periodically
    negative = -(rng.random((500, 3)) * np.float32(1e-3)).astype(np.float32)  # just below 0
    huge = (rng.random((50, 3)) * 4e9 - 2e9).astype(np.float32)               # |x| >= 2^30: FP64 path
    tiny = (rng.random((500, 3)) * 1e-30).astype(np.float32)                  # offsets that round
    pos = np.concatenate([faces, edge, dup, outside, negative, huge, tiny])
    pos = pos[rng.permutation(len(pos))]
    _assert_bit_exact(pos, 1.0, K)


def test_bin_one_cell_holds_everything_and_empty_regions():
    pos = np.full((5000, 3), 0.51, np.float32)
    _assert_bit_exact(pos, 1.0, 9)
    half = uniform_positions(20000, 11) * np.float32(0.5)   # upper half of the box empty
    _assert_bit_exact(half, 1.0, 16)


def test_bin_clustered_large_cells():
    pos = clustered_positions(200000, 6, 12, n_sph=20)
    _assert_bit_exact(pos, 1.0, 6)


def test_bin_nonfinite_sets_status():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    pos = uniform_positions(1000, 3)
    dev = torch.from_numpy(pos).cuda()
    nf.forces(dev, 1.0, 8, 2, 1e-3)
    assert nf.status() == _lib.NF_OK
    pos[17, 1] = np.nan
    pos[900, 2] = np.inf
    nf.forces(torch.from_numpy(pos).cuda(), 1.0, 8, 2, 1e-3)
    assert nf.status() == _lib.NF_ERR_NONFINITE
    nf.forces(dev, 1.0, 8, 2, 1e-3)
    assert nf.status() == _lib.NF_OK   # cleared by the next call
