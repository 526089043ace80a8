"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments on the host before launching."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2110_11392_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nf.h")

# fake, never dereferenced: every call below must fail validation first
FAKE = ctypes.c_void_p(0x7F0000001000)
FAKE_WS = ctypes.c_void_p(0x7F0000100000)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nf_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported():
    lib = _lib.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), f"{n} declared in nf.h but not exported"
    assert set(names) == set(_lib.exported_symbols())


def test_version_and_default_tuning():
    assert "sm_103a" in _lib.nf_version()
    assert _lib.nf_get_default_tuning() == (4, 128, 8, 0)
    assert _lib.nf_get_default_tuning_adjoint() == (4, 128, 8, 1)
    # setting the default sets both directions; the adjoint's can then differ; NULL restores both
    _lib.nf_set_default_tuning((2, 64, 4, 0))
    assert _lib.nf_get_default_tuning() == (2, 64, 4, 0) == _lib.nf_get_default_tuning_adjoint()
    _lib.nf_set_default_tuning_adjoint((3, 128, 8, 0))
    assert _lib.nf_get_default_tuning() == (2, 64, 4, 0)
    assert _lib.nf_get_default_tuning_adjoint() == (3, 128, 8, 0)
    with pytest.raises(_lib.NFError):
        _lib.nf_set_default_tuning_adjoint((3, 96, 8, 0))
    _lib.nf_set_default_tuning(None)
    assert _lib.nf_get_default_tuning() == (4, 128, 8, 0)
    assert _lib.nf_get_default_tuning_adjoint() == (4, 128, 8, 1)


def test_workspace_bytes():
    a = _lib.nf_workspace_bytes(32768, 8, 2)
    b = _lib.nf_workspace_bytes(2 * 32768, 8, 2)
    assert 0 < a < b
    assert _lib.nf_workspace_bytes(1000, 4, 2) == 0    # K < 2R+1
    assert _lib.nf_workspace_bytes(0, 8, 2) == 0       # N < 1
    assert _lib.nf_workspace_bytes(1000, 8, 5) == 0    # R > NF_MAX_R
    assert _lib.nf_workspace_bytes(1000, 1291, 2) == 0  # K^3 >= 2^31


def _forces(N=1000, box=1.0, K=8, R=2, eps=1e-3, pos=FAKE, acc=FAKE, ws=FAKE_WS, ws_bytes=1 << 40):
    lib = _lib.load()
    return lib.nf_forces(pos, N, box, K, R, eps, acc, None, ws, ws_bytes, None)


@pytest.mark.parametrize("kw,code", [
    (dict(K=4, R=2), _lib.NF_ERR_ARG),            # stencil wraps onto itself
    (dict(N=0), _lib.NF_ERR_ARG),
    (dict(N=-5), _lib.NF_ERR_ARG),
    (dict(N=1 << 31), _lib.NF_ERR_ARG),
    (dict(box=0.0), _lib.NF_ERR_ARG),
    (dict(box=-1.0), _lib.NF_ERR_ARG),
    (dict(box=float("nan")), _lib.NF_ERR_ARG),
    (dict(eps=0.0), _lib.NF_ERR_ARG),
    (dict(eps=float("inf")), _lib.NF_ERR_ARG),
    (dict(eps=0.25 / 2.16 + 1e-9, K=8, R=2), _lib.NF_ERR_ARG),   # eps_s > R w
    (dict(eps=1e-9), _lib.NF_ERR_ARG),            # eps_s < 1e-5 w
    (dict(R=0), _lib.NF_ERR_ARG),
    (dict(R=5, K=11), _lib.NF_ERR_ARG),
    (dict(pos=None), _lib.NF_ERR_ARG),
    (dict(acc=None), _lib.NF_ERR_ARG),
    (dict(ws=None), _lib.NF_ERR_WORKSPACE),
    (dict(ws_bytes=100), _lib.NF_ERR_WORKSPACE),
    (dict(ws=ctypes.c_void_p(0x7F0000100010)), _lib.NF_ERR_WORKSPACE),  # misaligned
])
def test_forces_rejects_bad_arguments(kw, code):
    assert _forces(**kw) == code
    assert _lib.nf_last_error() != ""


def test_largest_valid_softening_passes_validation_only_to_workspace_check():
    # eps_s exactly at R w is allowed; the call then stops at the workspace check
    assert _forces(eps=0.25 / 2.16 * (1 - 1e-12), ws_bytes=16) == _lib.NF_ERR_WORKSPACE


def test_adjoint_and_bin_reject_bad_arguments():
    lib = _lib.load()
    assert lib.nf_forces_adjoint(FAKE, None, 1000, 1.0, 8, 2, 1e-3, FAKE, FAKE_WS, 1 << 40, None) == _lib.NF_ERR_ARG
    assert lib.nf_bin(FAKE, 1000, 1.0, 0, FAKE, FAKE, FAKE, FAKE_WS, 1 << 40, None) == _lib.NF_ERR_ARG
    assert lib.nf_bin(FAKE, 1000, 1.0, 8, FAKE, ctypes.c_void_p(0x7F0000001004), FAKE, FAKE_WS, 1 << 40,
                      None) == _lib.NF_ERR_ARG  # rel not 16-byte aligned
    assert lib.nf_bin(FAKE, 1000, 1.0, 8, FAKE, FAKE, FAKE, FAKE_WS, 64, None) == _lib.NF_ERR_WORKSPACE


def test_batched_rejects_bad_packing_and_tuning():
    lib = _lib.load()
    boxes = [dict(N=100, K=5, R=2, eps=1e-3), dict(N=200, K=6, R=2, eps=1e-3)]
    arr = _lib.make_boxes(boxes)
    arr[1].pos_offset = 99
    assert lib.nf_forces_batched(arr, 2, FAKE, FAKE, None, None, FAKE_WS, 1 << 40, None) == _lib.NF_ERR_ARG
    assert "packed" in _lib.nf_last_error()
    arr = _lib.make_boxes(boxes)
    bad = _lib.nf_tuning(5, 128, 8, 0)
    assert lib.nf_forces_batched(arr, 2, FAKE, FAKE, None, ctypes.byref(bad), FAKE_WS, 1 << 40,
                                 None) == _lib.NF_ERR_ARG
    assert lib.nf_forces_batched(arr, 0, FAKE, FAKE, None, None, FAKE_WS, 1 << 40, None) == _lib.NF_ERR_ARG
    assert _lib.nf_workspace_bytes_batched(boxes) > 0
    with pytest.raises(_lib.NFError):
        _lib.nf_set_default_tuning((4, 96, 8, 0))
    assert _lib.nf_get_default_tuning() == (4, 128, 8, 0)


def test_status_read_rejects_null_workspace():
    assert _lib.load().nf_status_read(None, None) == _lib.NF_ERR_WORKSPACE


def test_workloads_are_seeded_and_exact():
    from workloads import clustered_positions, config_batched, uniform_positions
    from workloads.recipes import sphere_counts
    a = clustered_positions(20000, 8, 7)
    b = clustered_positions(20000, 8, 7)
    assert np.array_equal(a, b) and a.dtype == np.float32
    assert a.min() >= 0 and a.max() < 1
    c = sphere_counts(12000, 40, np.random.Generator(np.random.PCG64(1)))
    assert c.sum() == 12000 and c.min() >= 20
    u = uniform_positions(1000, 3)
    assert np.array_equal(u, uniform_positions(1000, 3))
    w = config_batched(nboxes=4)
    assert sum(bx["N"] for bx in w.boxes) == w.N
    assert all(bx["K"] >= 5 for bx in w.boxes)


def test_far_field_sizes_and_host_checks():
    lib = _lib.load()
    nt = lambda p: (p + 3) * (p + 2) * (p + 1) // 6
    for K, p in [(5, 0), (8, 8), (11, 8), (32, 12)]:
        b = _lib.nf_derivatives_bytes(K, p)
        assert b >= 8 * nt(p) * K * K * (K // 2 + 1) + 256   # one real per (term, frequency)
        assert b % 256 == 0
        assert _lib.nf_far_workspace_bytes(1000, K, p) > 8 * nt(p) * K ** 3
    assert _lib.nf_derivatives_bytes(8, 13) == 0 and _lib.nf_derivatives_bytes(0, 4) == 0
    # 165 terms x 236^3 cells would overflow the FFT plans' 32-bit offsets; 235^3 does not
    assert _lib.nf_derivatives_bytes(236, 8) == 0 and _lib.nf_derivatives_bytes(235, 8) > 0
    assert _lib.nf_far_workspace_bytes(0, 8, 4) == 0
    big = 1 << 40
    # rejected on the host before anything is launched
    for K, R, p, box in [(4, 2, 4, 1.0), (8, 0, 4, 1.0), (8, 2, 13, 1.0), (8, 2, -1, 1.0), (8, 2, 4, 0.0)]:
        assert lib.nf_derivatives(K, R, p, box, FAKE_WS, big, FAKE_WS, big, None) == _lib.NF_ERR_ARG
    assert lib.nf_derivatives(8, 2, 4, 1.0, None, big, FAKE_WS, big, None) == _lib.NF_ERR_ARG
    assert lib.nf_derivatives(8, 2, 4, 1.0, FAKE_WS, 100, FAKE_WS, big, None) == _lib.NF_ERR_WORKSPACE
    assert lib.nf_far_forces(FAKE, 1000, 1.0, 4, 2, 4, FAKE_WS, big, None, None, None, FAKE_WS, big,
                             None) == _lib.NF_ERR_ARG
    assert lib.nf_far_forces(FAKE, 1000, 1.0, 8, 2, 4, FAKE_WS, 100, None, None, None, FAKE_WS, big,
                             None) == _lib.NF_ERR_ARG
    assert lib.nf_far_forces(FAKE, 1000, 1.0, 8, 2, 4, FAKE_WS, big, None, None, None, FAKE_WS, 4096,
                             None) == _lib.NF_ERR_WORKSPACE


def test_far_arith_switch_on_host():
    lib = _lib.load()
    before = lib.nf_far_get_arith()
    assert before in (_lib.NF_FAR_FP64, _lib.NF_FAR_DOUBLE_FLOAT)
    assert lib.nf_far_set_arith(5) == _lib.NF_ERR_ARG
    assert lib.nf_far_set_arith(_lib.NF_FAR_FP64) == _lib.NF_OK and lib.nf_far_get_arith() == _lib.NF_FAR_FP64
    assert lib.nf_far_set_arith(before) == _lib.NF_OK


def test_density_mode_switch_on_host():
    lib = _lib.load()
    assert lib.nf_get_density_mode() == _lib.NF_DENS_AUTO
    assert lib.nf_set_density_mode(3) == _lib.NF_ERR_ARG
    assert lib.nf_set_density_mode(-1) == _lib.NF_ERR_ARG
    assert lib.nf_get_density_mode() == _lib.NF_DENS_AUTO
    for m in (_lib.NF_DENS_FUSED, _lib.NF_DENS_DEFERRED, _lib.NF_DENS_AUTO):
        assert lib.nf_set_density_mode(m) == _lib.NF_OK and lib.nf_get_density_mode() == m
