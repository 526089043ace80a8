"""nf_forces_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a plugin whose host program owns every device allocation
through its own pool, or code that must not allocate while work is being
captured) cannot hand the library a workspace, so this entry point runs
nf_forces on a fixed scratch array built into the library.  The test checks,
through the C ABI, that calls in a row give exactly the forces and net force of
nf_forces with a caller workspace (both run the same kernels with the same
tuning, so the results must be bit-identical), including a small problem run
again after a larger one has left its contents in the shared array, that the
first result also meets the oracle parity bar, and that problems too large for
the array are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2110_11392_gb300 import _lib
from workloads import config_plain, uniform_positions
from workloads.recipes import Workload

from _helpers import FORCE_MAX, FORCE_MEDIAN, frac_stats


def test_noalloc_rejects_problems_larger_than_its_array():
    import ctypes
    fake = ctypes.c_void_p(0x7F0000001000)
    # 2^21 particles need far more than the fixed scratch array: refused on the host
    rc = _lib.load().nf_forces_noalloc(fake, 1 << 21, 1.0, 32, 2, 1e-4, fake, None, None)
    assert rc == _lib.NF_ERR_WORKSPACE
    assert "nf_forces_noalloc" in _lib.nf_last_error()
    rc = _lib.load().nf_forces_noalloc(fake, 1000, 1.0, 4, 2, 1e-3, fake, None, None)
    assert rc == _lib.NF_ERR_ARG


@pytest.mark.gpu
def test_noalloc_matches_nf_forces_on_calls_in_a_row():
    import torch
    import oracle
    first = config_plain()                                    # 32^3 particles, K = 8
    second = Workload("second", uniform_positions(50000, 77), 1.0, 9, 2, 1.0 / (40 * 50000 ** (1 / 3)))
    # the small box again after the larger one: the array holds the larger call's leftovers
    for q, w in enumerate((first, second, first)):
        pos = torch.from_numpy(w.pos).cuda()
        ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device="cuda")
        ref = torch.empty_like(pos)
        ref_net = torch.empty(3, dtype=torch.float64, device="cuda")
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, ref, ref_net, ws)
        out = torch.full_like(pos, float("nan"))
        net = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.nf_forces_noalloc(pos, w.box, w.K, w.R, w.eps, out, net)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"call {q} ({w.name}): forces differ from nf_forces"
        assert torch.equal(net, ref_net), f"call {q} ({w.name}): net force differs from nf_forces"
        if q == 0:
            a = out.cpu().numpy()
            med, _, mx = frac_stats(a, oracle.forces(w.pos, w.box, w.K, w.R, w.eps))
            assert med <= FORCE_MEDIAN and mx <= FORCE_MAX, (w.name, med, mx)
