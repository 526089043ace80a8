"""The autotuner (autotune.tune) and the batched runner that uses it.

The tuner times each candidate tuning (sinks per lane, stage, warps per block,
blocks per SM) on the caller's boxes and returns the fastest; the checks here
are that its pick is the minimum of its own timings, that the cache returns
the same record without timing again, that BatchedNearField(tune="auto") uses
the pick, and that the picked tuning gives per box exactly what nf_forces gives
with that tuning as the library default, at the oracle parity bar.
"""
import json

import numpy as np
import pytest

import oracle
from workloads import config_batched
from workloads.recipes import Workload

from _helpers import assert_force_parity, sample_sinks, to_dev

pytestmark = pytest.mark.gpu

CANDS = [(2, 128, 8, 0), (1, 64, 8, 3), (4, 128, 4, 0)]


def _key(t):
    return ",".join(map(str, t))


def test_tuner_pick_cache_and_parity(tmp_path):
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib, autotune
    w = config_batched(nboxes=6, seed=11)
    pos = to_dev(w.pos)
    cache = str(tmp_path / "tuning.json")
    best, ms = autotune.tune(w.boxes, pos, candidates=CANDS, reps=2, cache=cache)
    assert set(ms) == {_key(t) for t in CANDS}
    assert all(v > 0 for v in ms.values())
    assert ms[_key(best)] == min(ms.values())
    rec = json.load(open(cache))
    assert len(rec) == 1 and list(rec.values())[0]["best"] == list(best)
    # the cache round-trips: the same pick and timings come back without timing again
    best2, ms2 = autotune.tune(w.boxes, pos, candidates=CANDS, reps=2, cache=cache)
    assert best2 == best and ms2 == ms
    # a different candidate list is not served from that record
    _, ms3 = autotune.tune(w.boxes, pos, candidates=CANDS[:2], reps=1, cache=cache)
    assert set(ms3) == {_key(t) for t in CANDS[:2]}
    # the runner with tune="auto" searches the default candidate list (its own cache file)
    run = nf.BatchedNearField(w.boxes, tune="auto", tune_cache=str(tmp_path / "auto.json"))
    acc = run(pos).clone()
    torch.cuda.synchronize()
    assert run.tune is not None and run.tune_timings is not None
    assert run.tune_timings[_key(run.tune)] == min(run.tune_timings.values())
    acc = acc.cpu().numpy()
    old, old_adj = _lib.nf_get_default_tuning(), _lib.nf_get_default_tuning_adjoint()
    _lib.nf_set_default_tuning(run.tune)
    try:
        off = 0
        for q, b in enumerate(w.boxes):
            bw = Workload("box", w.pos[off:off + b["N"]], b["box"], b["K"], b["R"], b["eps"])
            single = nf.forces(to_dev(bw.pos), bw.box, bw.K, bw.R, bw.eps)
            a = acc[off:off + bw.N]
            assert np.array_equal(a, single.cpu().numpy()), f"box {q}: tuned batch differs from nf_forces"
            idx = sample_sinks(bw, 300, seed=q)
            ref = oracle.forces(bw.pos, bw.box, bw.K, bw.R, bw.eps, sinks=idx)
            assert_force_parity(a[idx], ref, label=f"box {q} with tuning {run.tune}")
            off += bw.N
    finally:
        _lib.nf_set_default_tuning(old)
        _lib.nf_set_default_tuning_adjoint(old_adj)


def test_auto_tuning_then_graph_capture(tmp_path):
    import torch
    import paper_2110_11392_gb300 as nf
    w = config_batched(nboxes=4, seed=12)
    pos = to_dev(w.pos)
    eager = nf.BatchedNearField(w.boxes, tune="auto", tune_cache=str(tmp_path / "t.json"))
    ref = eager(pos).clone()
    g = nf.BatchedNearField(w.boxes, tune="auto", tune_cache=str(tmp_path / "t.json"))
    g.pos.copy_(pos)
    g.capture()  # the search (here: the cached record) runs before the capture
    assert g.tune == eager.tune
    out = g()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_tune_rejects_unknown_mode():
    import paper_2110_11392_gb300 as nf
    w = config_batched(nboxes=2, seed=13)
    with pytest.raises(ValueError):
        nf.BatchedNearField(w.boxes, tune="fastest")
