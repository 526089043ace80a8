"""Debug mode: guard blocks after every workspace region (a stand-in for a
memory checker).  Every entry point leaves them intact; a planted overwrite
(from the host, between calls) is reported as NF_ERR_CORRUPT."""
import numpy as np
import pytest

from paper_2110_11392_gb300 import _lib
from workloads import config_plain

from _helpers import to_dev


def test_debug_mode_grows_the_workspace():
    base = _lib.nf_workspace_bytes(32768, 8, 2)
    _lib.nf_set_debug(True)
    try:
        assert _lib.nf_workspace_bytes(32768, 8, 2) > base
    finally:
        _lib.nf_set_debug(False)
    assert _lib.nf_workspace_bytes(32768, 8, 2) == base


@pytest.mark.gpu
def test_guards_stay_intact_and_catch_an_overwrite():
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_plain()
    _lib.nf_set_debug(True)
    try:
        ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device="cuda")
        pos = to_dev(w.pos)
        acc = torch.empty_like(pos)
        g = torch.ones_like(pos)
        grad = torch.empty_like(pos)
        rho = torch.empty(w.N, dtype=torch.float32, device="cuda")
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
        assert _lib.nf_status_read(ws) == _lib.NF_OK
        _lib.nf_forces_adjoint(pos, g, w.box, w.K, w.R, w.eps, grad, ws)
        assert _lib.nf_status_read(ws) == _lib.NF_OK
        _lib.nf_forces_density(pos, w.box, w.K, w.R, w.eps, 0.5 / w.K, acc, rho, ws)
        assert _lib.nf_status_read(ws) == _lib.NF_OK
        M = torch.empty((w.K ** 3, 165), dtype=torch.float64, device="cuda")
        _lib.nf_multipoles(pos, w.box, w.K, 8, M, ws)
        assert _lib.nf_status_read(ws) == _lib.NF_OK
        dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
        vel = torch.zeros_like(pos)
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
        _lib.nf_kdk_step(pos, vel, acc, w.box, w.K, w.R, w.eps, dt, _lib.make_step_params(0.25), ws)
        assert _lib.nf_status_read(ws) == _lib.NF_OK
        # the results are those of the normal build
        plain = nf.forces(pos, w.box, w.K, w.R, w.eps)
        _lib.nf_forces(pos, w.box, w.K, w.R, w.eps, acc, None, ws)
        assert torch.equal(acc, plain)
        # plant an overwrite in the first guard block, which follows the
        # 256-byte status header at the start of every workspace
        ws[256 + 17] = 0
        _lib.nf_debug_check(ws)
        assert _lib.nf_status_read(ws) == _lib.NF_ERR_CORRUPT
    finally:
        _lib.nf_set_debug(False)


@pytest.mark.gpu
def test_far_field_entries_keep_their_guards():
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_plain()
    pos = to_dev(w.pos)
    ff = nf.FarField(w.K, w.R, 6, w.box)
    # reference results of the normal build
    ref_far = ff(pos)
    ref_tot = ff.total(pos, w.eps).clone()
    torch.cuda.synchronize()
    _lib.nf_set_debug(True)
    try:
        ws = torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device="cuda")
        wsf = torch.empty(_lib.nf_far_workspace_bytes(w.N, w.K, 6), dtype=torch.uint8, device="cuda")
        # a far workspace that has never been binned must not confuse the guard check
        wsf.fill_(0xAB)
        far = torch.empty((w.N, 3), dtype=torch.float64, device="cuda")
        tot = torch.empty_like(pos)
        _lib.nf_forces_total(pos, w.box, w.K, w.R, w.eps, 6, ff.derivs, tot, ws, wsf)
        assert _lib.nf_status_read(wsf) == _lib.NF_OK and _lib.nf_status_read(ws) == _lib.NF_OK
        _lib.nf_far_forces(pos, w.box, w.K, w.R, 6, ff.derivs, far, None, None, wsf)
        assert _lib.nf_status_read(wsf) == _lib.NF_OK
        vel = torch.zeros_like(pos)
        acc = tot.clone()
        dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
        _lib.nf_kdk_step_far(pos.clone(), vel, acc, w.box, w.K, w.R, w.eps, 6, ff.derivs, dt, None, ws, wsf)
        assert _lib.nf_status_read(wsf) == _lib.NF_OK and _lib.nf_status_read(ws) == _lib.NF_OK
        assert torch.equal(far, ref_far) and torch.equal(tot, ref_tot)
        # an overwrite in the last guard (after the last far-field region) is caught
        wsf[wsf.numel() - 100] = 0
        _lib.nf_debug_check(wsf)
        assert _lib.nf_status_read(wsf) == _lib.NF_ERR_CORRUPT
    finally:
        _lib.nf_set_debug(False)
