"""The 512^3 clustered box (134,217,728 particles, K = 128) at full size: binning
bit-exact against the oracle, and forces on sampled sinks (the oracle computes
them one by one), through the same nf_forces call the benchmark times."""
import numpy as np
import pytest

import oracle
from workloads import config_large

from _helpers import assert_force_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def large():
    return config_large()


def test_large_binning_bit_exact(large):
    import torch
    import paper_2110_11392_gb300 as nf
    w = large
    pos = torch.from_numpy(w.pos).cuda()
    off, rel, perm = nf.bin_particles(pos, w.box, w.K)
    torch.cuda.synchronize()
    off_o, rel_o, perm_o = oracle.bin_particles(w.pos, w.box, w.K)
    assert np.array_equal(off.cpu().numpy(), off_o)
    assert np.array_equal(perm.cpu().numpy(), perm_o)
    assert np.array_equal(rel.cpu().numpy().view(np.int32), rel_o.view(np.int32))
    del pos, off, rel, perm
    torch.cuda.empty_cache()


def test_large_forces_sampled(large):
    import torch
    import paper_2110_11392_gb300 as nf
    w = large
    pos = torch.from_numpy(w.pos).cuda()
    acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
    torch.cuda.synchronize()
    rng = np.random.default_rng(22)
    idx = np.sort(rng.choice(w.N, 3000, replace=False))
    # add the particles of the densest cell, where FP32 accumulation is hardest
    off, _, perm = oracle.bin_particles(w.pos, w.box, w.K)
    c = int(np.argmax(np.diff(off)))
    idx = np.union1d(idx, perm[off[c]:off[c + 1]])
    a = acc[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.forces(w.pos, w.box, w.K, w.R, w.eps, sinks=idx)
    assert_force_parity(a, ref, label="512^3 sampled")
    del pos, acc
    torch.cuda.empty_cache()
