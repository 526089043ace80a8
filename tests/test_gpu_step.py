"""nf_kdk_step / nf_timestep: KDK leapfrog and Eq. (timestep) on the device,
against the FP64 oracle step and criterion."""
import numpy as np
import pytest

import oracle
from workloads import config_plain

from _helpers import assert_force_parity, to_dev

pytestmark = pytest.mark.gpu

ETA = 0.25


def _state(seed=5, N=32768, K=8):
    w = config_plain(N=N, K=K, seed=seed)
    rng = np.random.default_rng(seed + 100)
    vel = (0.02 * rng.standard_normal((w.N, 3))).astype(np.float32)
    return w, vel


def _ws(w):
    import torch
    from paper_2110_11392_gb300 import _lib
    return torch.empty(_lib.nf_workspace_bytes(w.N, w.K, w.R), dtype=torch.uint8, device="cuda")


def test_timestep_matches_oracle():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w, vel = _state()
    pos = to_dev(w.pos)
    acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = _ws(w)
    _lib.nf_timestep(pos, to_dev(vel), acc, w.box, w.K, _lib.make_step_params(ETA), dt, ws)
    cell = oracle.cell_of(w.pos, w.box, w.K)
    ref = oracle.timestep(vel, acc.cpu().numpy().astype(np.float64), cell, ETA)
    assert dt.item() == pytest.approx(ref, rel=1e-5)
    # the Hubble limit binds exactly when it is the smaller term
    _lib.nf_timestep(pos, to_dev(vel), acc, w.box, w.K, _lib.make_step_params(ETA, 1e-9, 1.0), dt, ws)
    assert dt.item() == 1e-9
    torch.cuda.synchronize()


def test_kdk_two_steps_match_oracle():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w, vel = _state(seed=6)
    pos, v = to_dev(w.pos), to_dev(vel)
    acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
    dt_val = 2e-3
    dt = torch.full((1,), dt_val, dtype=torch.float64, device="cuda")
    ws = _ws(w)
    xo, vo, ao = w.pos, vel, oracle.forces(w.pos, w.box, w.K, w.R, w.eps)
    for _ in range(2):
        _lib.nf_kdk_step(pos, v, acc, w.box, w.K, w.R, w.eps, dt, None, ws)
        xo, vo, ao = oracle.kdk_step(xo, vo, ao, dt_val, w.box, w.K, w.R, w.eps)
    torch.cuda.synchronize()
    xg, vg, ag = pos.cpu().numpy(), v.cpu().numpy(), acc.cpu().numpy()
    dx = (xg.astype(np.float64) - xo + 0.5) % 1.0 - 0.5
    assert np.abs(dx).max() < 1e-6            # FP32 state, a few roundings per step
    dv = np.linalg.norm(vg - vo, axis=1) / np.linalg.norm(vo, axis=1)
    assert np.median(dv) < 1e-6 and dv.max() < 1e-3
    # the accelerations after the step are the near-field forces at the new positions
    assert_force_parity(ag, oracle.forces(xg, w.box, w.K, w.R, w.eps), label="after 2 steps")


def test_kdk_reversible_and_momentum():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w, vel = _state(seed=7)
    pos, v = to_dev(w.pos), to_dev(vel)
    acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
    ws = _ws(w)
    p0 = vel.astype(np.float64).sum(axis=0)
    dtp = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    dtm = torch.full((1,), -1e-3, dtype=torch.float64, device="cuda")
    _lib.nf_kdk_step(pos, v, acc, w.box, w.K, w.R, w.eps, dtp, None, ws)
    moved = pos.cpu().numpy()
    p1 = v.cpu().numpy().astype(np.float64).sum(axis=0)
    _lib.nf_kdk_step(pos, v, acc, w.box, w.K, w.R, w.eps, dtm, None, ws)
    torch.cuda.synchronize()
    back = pos.cpu().numpy()
    assert np.abs(moved - w.pos).max() > 1e-5
    dx = (back.astype(np.float64) - w.pos + 0.5) % 1.0 - 0.5
    assert np.abs(dx).max() < 1e-6
    assert np.abs(v.cpu().numpy() - vel).max() < 1e-5 * np.abs(vel).max()
    assert np.abs(p1 - p0).max() < 1e-6 * np.abs(vel).sum()


def test_adaptive_loop_in_a_cuda_graph_is_bit_identical():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w, vel = _state(seed=8, N=20000, K=7)
    prm = _lib.make_step_params(ETA)

    def fresh():
        pos, v = to_dev(w.pos), to_dev(vel)
        acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        ws = _ws(w)
        _lib.nf_timestep(pos, v, acc, w.box, w.K, prm, dt, ws)
        return pos, v, acc, dt, ws

    pos, v, acc, dt, ws = fresh()
    for _ in range(4):
        _lib.nf_kdk_step(pos, v, acc, w.box, w.K, w.R, w.eps, dt, prm, ws)
    eager = (pos.clone(), v.clone(), acc.clone(), dt.clone())

    pos, v, acc, dt, ws = fresh()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(4):
            _lib.nf_kdk_step(pos, v, acc, w.box, w.K, w.R, w.eps, dt, prm, ws, stream=s)
    # capture does not run the work: start again from the initial state and replay
    pos.copy_(to_dev(w.pos))
    v.copy_(to_dev(vel))
    acc.copy_(nf.forces(pos, w.box, w.K, w.R, w.eps))
    _lib.nf_timestep(pos, v, acc, w.box, w.K, prm, dt, ws)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip((pos, v, acc, dt), eager):
        assert torch.equal(a, b)
    assert 0 < dt.item() < 1.0


def test_kdk_with_far_field_matches_oracle():
    # total force (near + far at order 4): two leapfrog steps against the oracle's
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w, vel = _state(seed=9)
    p = 4
    ff = nf.FarField(w.K, w.R, p, w.box)
    pos, v = to_dev(w.pos), to_dev(vel)
    acc = nf.forces(pos, w.box, w.K, w.R, w.eps)
    ff(pos, add_to=acc, want_far=False)
    dt_val = 2e-3
    dt = torch.full((1,), dt_val, dtype=torch.float64, device="cuda")
    ws = _ws(w)
    wsf = ff.workspace(w.N)
    D = oracle.derivatives(w.K, w.R, p, w.box)
    xo, vo = w.pos, vel
    ao = oracle.forces(w.pos, w.box, w.K, w.R, w.eps) + oracle.far_field(w.pos, w.box, w.K, w.R, p, D=D)
    for _ in range(2):
        _lib.nf_kdk_step_far(pos, v, acc, w.box, w.K, w.R, w.eps, p, ff.derivs, dt, None, ws, wsf)
        xo, vo, ao = oracle.kdk_step(xo, vo, ao, dt_val, w.box, w.K, w.R, w.eps, far_order=p, D=D)
    torch.cuda.synchronize()
    xg, vg, ag = pos.cpu().numpy(), v.cpu().numpy(), acc.cpu().numpy()
    dx = (xg.astype(np.float64) - xo + 0.5) % 1.0 - 0.5
    assert np.abs(dx).max() < 1e-6
    dv = np.linalg.norm(vg - vo, axis=1) / np.linalg.norm(vo, axis=1)
    assert np.median(dv) < 1e-6 and dv.max() < 1e-3
    ref = oracle.forces(xg, w.box, w.K, w.R, w.eps) + oracle.far_field(xg, w.box, w.K, w.R, p, D=D)
    assert_force_parity(ag, ref, label="near + far after 2 steps")
    # the adaptive form writes the next step's dt from the same criterion
    prm = _lib.make_step_params(ETA)
    _lib.nf_kdk_step_far(pos, v, acc, w.box, w.K, w.R, w.eps, p, ff.derivs, dt, prm, ws, wsf)
    torch.cuda.synchronize()
    cell = oracle.cell_of(pos.cpu().numpy(), w.box, w.K)
    ref_dt = oracle.timestep(v.cpu().numpy(), acc.cpu().numpy().astype(np.float64), cell, ETA)
    assert dt.item() == pytest.approx(ref_dt, rel=1e-5)
