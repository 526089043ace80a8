"""nf_forces_batched: box by box against nf_forces, against the oracle, and as a CUDA graph."""
import numpy as np
import pytest

import oracle
from workloads import config_batched, upstream_gradient
from workloads.recipes import Workload

from _helpers import assert_force_parity, sample_sinks, to_dev

pytestmark = pytest.mark.gpu


def _split(w):
    out, off = [], 0
    for b in w.boxes:
        out.append(Workload("box", w.pos[off:off + b["N"]], b["box"], b["K"], b["R"], b["eps"]))
        off += b["N"]
    return out


@pytest.mark.slow
def test_batched_equals_per_box_and_oracle():
    """The full batched workload (64 boxes, N log-uniform in [16^3, 96^3], the
    mix the benchmark times): every box equals nf_forces bit for bit and meets
    the oracle parity bar on sampled sinks."""
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_batched()
    assert len(w.boxes) == 64
    run = nf.BatchedNearField(w.boxes, net=True)
    acc = run(to_dev(w.pos)).clone()
    net = run.net.clone()
    torch.cuda.synchronize()
    acc = acc.cpu().numpy()
    off = 0
    for q, bw in enumerate(_split(w)):
        single, snet = nf.forces(to_dev(bw.pos), bw.box, bw.K, bw.R, bw.eps, net=True)
        a = acc[off:off + bw.N]
        assert np.array_equal(a, single.cpu().numpy()), f"box {q} differs from nf_forces"
        assert np.array_equal(net[q].cpu().numpy(), snet.cpu().numpy())
        idx = sample_sinks(bw, 500, seed=q)
        ref = oracle.forces(bw.pos, bw.box, bw.K, bw.R, bw.eps, sinks=idx)
        assert_force_parity(a[idx], ref, label=f"box {q}")
        off += bw.N


def test_graph_replay_is_bit_identical():
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_batched(nboxes=6, seed=9)
    eager = nf.BatchedNearField(w.boxes)
    ref = eager(to_dev(w.pos)).clone()
    g = nf.BatchedNearField(w.boxes).capture()
    for _ in range(3):
        out = g(to_dev(w.pos))
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # new inputs through the same graph
    w2 = config_batched(nboxes=6, seed=9)
    pos2 = w2.pos.copy()
    pos2[::7] = (pos2[::7] + np.float32(0.01)) % np.float32(1.0)
    out2 = g(to_dev(pos2)).clone()
    ref2 = eager(to_dev(pos2))
    torch.cuda.synchronize()
    assert torch.equal(out2, ref2)


def test_batched_adjoint_equals_per_box():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    w = config_batched(nboxes=4, seed=3)
    g = upstream_gradient(w.N, 5)
    arr = _lib.make_boxes(w.boxes)
    ws = torch.empty(_lib.nf_workspace_bytes_batched(w.boxes), dtype=torch.uint8, device="cuda")
    pos = to_dev(w.pos)
    grad = torch.empty_like(pos)
    _lib.nf_forces_adjoint_batched(arr, pos, to_dev(g), grad, None, ws)
    grad = grad.cpu().numpy()
    off = 0
    for bw in _split(w):
        single = nf.forces_adjoint(to_dev(bw.pos), to_dev(g[off:off + bw.N]), bw.box, bw.K, bw.R, bw.eps)
        assert np.array_equal(grad[off:off + bw.N], single.cpu().numpy())
        off += bw.N
