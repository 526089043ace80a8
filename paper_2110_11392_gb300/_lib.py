"""ctypes binding of libnf's C ABI (include/nf.h), one Python function per entry point.

The functions keep the C names and only marshal arguments: torch tensors are
passed as device pointers, the current CUDA stream as a handle.  All work runs
in libnf's kernels; nothing here computes.  If the library is missing or fails
to load, importing this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

from . import _build

NF_OK, NF_ERR_ARG, NF_ERR_CUDA, NF_ERR_WORKSPACE, NF_ERR_NONFINITE, NF_ERR_TIMEOUT, NF_ERR_CORRUPT = range(7)
NF_MAX_R = 4
STATUS_NAMES = {0: "NF_OK", 1: "NF_ERR_ARG", 2: "NF_ERR_CUDA", 3: "NF_ERR_WORKSPACE",
                4: "NF_ERR_NONFINITE", 5: "NF_ERR_TIMEOUT", 6: "NF_ERR_CORRUPT"}


class NFError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class nf_box(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("pos_offset", ctypes.c_int64), ("box", ctypes.c_double),
                ("eps", ctypes.c_double), ("K", ctypes.c_int), ("R", ctypes.c_int)]


class nf_profile(ctypes.Structure):
    _fields_ = [("bin_ms", ctypes.c_double), ("worklist_ms", ctypes.c_double), ("pair_ms", ctypes.c_double),
                ("combine_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class nf_far_profile(ctypes.Structure):
    _fields_ = [("bin_ms", ctypes.c_double), ("multipoles_ms", ctypes.c_double),
                ("convolution_ms", ctypes.c_double), ("taylor_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class nf_step_params(ctypes.Structure):
    _fields_ = [("eta_acc", ctypes.c_double), ("eta_h", ctypes.c_double), ("hubble", ctypes.c_double)]


class nf_tuning(ctypes.Structure):
    _fields_ = [("sinks_per_lane", ctypes.c_int), ("stage", ctypes.c_int),
                ("warps_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int)]

    def as_tuple(self):
        return (self.sinks_per_lane, self.stage, self.warps_per_block, self.blocks_per_sm)


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> ctypes.CDLL:
    """Load libnf.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build_library()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libnf.so not found at {_build.LIB}; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    P, i64, i32, f64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "nf_last_error": (ctypes.c_char_p, []),
        "nf_version": (ctypes.c_char_p, []),
        "nf_workspace_bytes": (sz, [i64, i32, i32]),
        "nf_workspace_bytes_batched": (sz, [P, i32]),
        "nf_bin": (i32, [P, i64, f64, i32, P, P, P, P, sz, P]),
        "nf_forces": (i32, [P, i64, f64, i32, i32, f64, P, P, P, sz, P]),
        "nf_forces_adjoint": (i32, [P, P, i64, f64, i32, i32, f64, P, P, sz, P]),
        "nf_forces_batched": (i32, [P, i32, P, P, P, P, P, sz, P]),
        "nf_forces_adjoint_batched": (i32, [P, i32, P, P, P, P, P, sz, P]),
        "nf_set_default_tuning": (i32, [P]),
        "nf_get_default_tuning": (None, [P]),
        "nf_set_default_tuning_adjoint": (i32, [P]),
        "nf_get_default_tuning_adjoint": (None, [P]),
        "nf_status_read": (i32, [P, P]),
        "nf_stats_read": (i32, [P, P, P]),
        "nf_stage_stats_read": (i32, [P, P, P]),
        "nf_profile_enable": (i32, [i32]),
        "nf_profile_read": (i32, [i32, P]),
        "nf_kernel_launches": (i64, []),
        "nf_forces_noalloc": (i32, [P, i64, f64, i32, i32, f64, P, P, P]),
        "nf_forces_density": (i32, [P, i64, f64, i32, i32, f64, f64, P, P, P, sz, P]),
        "nf_timestep": (i32, [P, P, P, i64, f64, i32, P, P, P, sz, P]),
        "nf_kdk_step": (i32, [P, P, P, i64, f64, i32, i32, f64, P, P, P, sz, P]),
        "nf_multipoles": (i32, [P, i64, f64, i32, i32, P, P, sz, P]),
        "nf_derivatives_bytes": (sz, [i32, i32]),
        "nf_far_workspace_bytes": (sz, [i64, i32, i32]),
        "nf_derivatives": (i32, [i32, i32, i32, f64, P, sz, P, sz, P]),
        "nf_far_forces": (i32, [P, i64, f64, i32, i32, i32, P, sz, P, P, P, P, sz, P]),
        "nf_far_profile_read": (i32, [i32, P]),
        "nf_far_release": (i32, []),
        "nf_far_set_arith": (i32, [i32]),
        "nf_far_get_arith": (i32, []),
        "nf_forces_total": (i32, [P, i64, f64, i32, i32, f64, i32, P, sz, P, P, sz, P, sz, P]),
        "nf_kdk_step_far": (i32, [P, P, P, i64, f64, i32, i32, f64, i32, P, sz, P, P, P, sz, P, sz, P]),
        "nf_set_debug": (i32, [i32]),
        "nf_set_density_mode": (i32, [i32]),
        "nf_get_density_mode": (i32, []),
        "nf_debug_check": (i32, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> Sequence[str]:
    return ("nf_last_error", "nf_version", "nf_workspace_bytes", "nf_workspace_bytes_batched",
            "nf_bin", "nf_forces", "nf_forces_adjoint", "nf_forces_batched",
            "nf_forces_adjoint_batched", "nf_set_default_tuning", "nf_get_default_tuning",
            "nf_set_default_tuning_adjoint", "nf_get_default_tuning_adjoint",
            "nf_status_read", "nf_stats_read", "nf_stage_stats_read", "nf_profile_enable", "nf_profile_read",
            "nf_kernel_launches", "nf_forces_noalloc", "nf_forces_density", "nf_timestep",
            "nf_kdk_step", "nf_multipoles", "nf_set_debug", "nf_debug_check",
            "nf_derivatives_bytes", "nf_far_workspace_bytes", "nf_derivatives", "nf_far_forces",
            "nf_far_profile_read", "nf_far_release", "nf_kdk_step_far", "nf_forces_total",
            "nf_far_set_arith", "nf_far_get_arith", "nf_set_density_mode", "nf_get_density_mode")


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, where: str):
    if rc != NF_OK:
        raise NFError(rc, where, load().nf_last_error().decode())


def nf_last_error() -> str:
    return load().nf_last_error().decode()


def nf_version() -> str:
    return load().nf_version().decode()


def nf_workspace_bytes(N: int, K: int, R: int) -> int:
    return int(load().nf_workspace_bytes(int(N), int(K), int(R)))


def make_boxes(boxes) -> "ctypes.Array":
    arr = (nf_box * len(boxes))()
    off = 0
    for i, b in enumerate(boxes):
        arr[i].N = int(b["N"])
        arr[i].pos_offset = int(b.get("pos_offset", off))
        arr[i].box = float(b.get("box", 1.0))
        arr[i].eps = float(b["eps"])
        arr[i].K = int(b["K"])
        arr[i].R = int(b.get("R", 2))
        off += int(b["N"])
    return arr


def nf_workspace_bytes_batched(boxes) -> int:
    arr = make_boxes(boxes)
    return int(load().nf_workspace_bytes_batched(arr, len(boxes)))


def make_tuning(t) -> Optional[nf_tuning]:
    if t is None:
        return None
    if isinstance(t, nf_tuning):
        return t
    s, b, w, n = t
    return nf_tuning(int(s), int(b), int(w), int(n))


def nf_bin(pos: torch.Tensor, box: float, K: int, cell_offsets: torch.Tensor, rel: torch.Tensor,
           perm: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_bin(_ptr(pos), pos.shape[0], float(box), int(K), _ptr(cell_offsets), _ptr(rel),
                         _ptr(perm), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "nf_bin")


def nf_forces(pos: torch.Tensor, box: float, K: int, R: int, eps: float, acc: torch.Tensor,
              net: Optional[torch.Tensor], ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_forces(_ptr(pos), pos.shape[0], float(box), int(K), int(R), float(eps), _ptr(acc),
                            _ptr(net), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "nf_forces")


def nf_forces_density(pos: torch.Tensor, box: float, K: int, R: int, eps: float, b: float,
                      acc: torch.Tensor, rho: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_forces_density(_ptr(pos), pos.shape[0], float(box), int(K), int(R), float(eps), float(b),
                                    _ptr(acc), _ptr(rho), _ptr(ws), ws.numel() * ws.element_size(),
                                    _stream(stream)),
           "nf_forces_density")


def nf_forces_adjoint(pos: torch.Tensor, g: torch.Tensor, box: float, K: int, R: int, eps: float,
                      grad: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_forces_adjoint(_ptr(pos), _ptr(g), pos.shape[0], float(box), int(K), int(R),
                                    float(eps), _ptr(grad), _ptr(ws), ws.numel() * ws.element_size(),
                                    _stream(stream)),
           "nf_forces_adjoint")


def nf_forces_batched(boxes_arr, pos_cat: torch.Tensor, acc_cat: torch.Tensor,
                      net: Optional[torch.Tensor], tune, ws: torch.Tensor, stream=None) -> None:
    t = make_tuning(tune)
    _check(load().nf_forces_batched(boxes_arr, len(boxes_arr), _ptr(pos_cat), _ptr(acc_cat), _ptr(net),
                                    ctypes.byref(t) if t is not None else None, _ptr(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)),
           "nf_forces_batched")


def nf_forces_adjoint_batched(boxes_arr, pos_cat: torch.Tensor, g_cat: torch.Tensor,
                              grad_cat: torch.Tensor, tune, ws: torch.Tensor, stream=None) -> None:
    t = make_tuning(tune)
    _check(load().nf_forces_adjoint_batched(boxes_arr, len(boxes_arr), _ptr(pos_cat), _ptr(g_cat),
                                            _ptr(grad_cat), ctypes.byref(t) if t is not None else None,
                                            _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "nf_forces_adjoint_batched")


def nf_set_default_tuning(tune) -> None:
    t = make_tuning(tune)
    _check(load().nf_set_default_tuning(ctypes.byref(t) if t is not None else None),
           "nf_set_default_tuning")


def nf_get_default_tuning() -> tuple:
    t = nf_tuning()
    load().nf_get_default_tuning(ctypes.byref(t))
    return t.as_tuple()


def nf_set_default_tuning_adjoint(tune) -> None:
    t = make_tuning(tune)
    _check(load().nf_set_default_tuning_adjoint(ctypes.byref(t) if t is not None else None),
           "nf_set_default_tuning_adjoint")


def nf_get_default_tuning_adjoint() -> tuple:
    t = nf_tuning()
    load().nf_get_default_tuning_adjoint(ctypes.byref(t))
    return t.as_tuple()


def nf_status_read(ws: torch.Tensor, stream=None) -> int:
    return int(load().nf_status_read(_ptr(ws), _stream(stream)))


def nf_stats_read(ws: torch.Tensor, stream=None) -> dict:
    out = (ctypes.c_int64 * 4)()
    _check(load().nf_stats_read(_ptr(ws), out, _stream(stream)), "nf_stats_read")
    return {"pairs": int(out[0]), "items": int(out[1]), "max_occupancy": int(out[2]),
            "lane_pairs": int(out[3])}


def nf_stage_stats_read(ws: torch.Tensor, stream=None) -> dict:
    out = (ctypes.c_int64 * 3)()
    _check(load().nf_stage_stats_read(_ptr(ws), out, _stream(stream)), "nf_stage_stats_read")
    return {"stages": int(out[0]), "exact": int(out[1]), "rerun": int(out[2])}


def nf_profile_enable(on: bool) -> None:
    _check(load().nf_profile_enable(1 if on else 0), "nf_profile_enable")


def nf_profile_read(back: int = 0) -> dict:
    p = nf_profile()
    _check(load().nf_profile_read(int(back), ctypes.byref(p)), "nf_profile_read")
    return {"bin_ms": p.bin_ms, "worklist_ms": p.worklist_ms, "pair_ms": p.pair_ms,
            "combine_ms": p.combine_ms, "total_ms": p.total_ms}


def nf_far_profile_read(back: int = 0) -> dict:
    p = nf_far_profile()
    _check(load().nf_far_profile_read(int(back), ctypes.byref(p)), "nf_far_profile_read")
    return {"bin_ms": p.bin_ms, "multipoles_ms": p.multipoles_ms, "convolution_ms": p.convolution_ms,
            "taylor_ms": p.taylor_ms, "total_ms": p.total_ms}


def nf_kernel_launches() -> int:
    return int(load().nf_kernel_launches())


def nf_forces_noalloc(pos: torch.Tensor, box: float, K: int, R: int, eps: float, acc: torch.Tensor,
                      net: Optional[torch.Tensor] = None, stream=None) -> None:
    """nf_forces without a workspace: the library's fixed scratch array is used
    instead (for callers that cannot allocate device memory; see include/nf.h)."""
    _check(load().nf_forces_noalloc(_ptr(pos), pos.shape[0], float(box), int(K), int(R), float(eps),
                                    _ptr(acc), _ptr(net), _stream(stream)),
           "nf_forces_noalloc")


def make_step_params(eta_acc: float, eta_h: float = 0.0, hubble: float = 0.0) -> nf_step_params:
    return nf_step_params(float(eta_acc), float(eta_h), float(hubble))


def nf_timestep(pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, box: float, K: int, prm,
                dt: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_timestep(_ptr(pos), _ptr(vel), _ptr(acc), pos.shape[0], float(box), int(K),
                              ctypes.byref(prm), _ptr(dt), _ptr(ws), ws.numel() * ws.element_size(),
                              _stream(stream)),
           "nf_timestep")


def nf_kdk_step(pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, box: float, K: int, R: int, eps: float,
                dt: torch.Tensor, prm, ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_kdk_step(_ptr(pos), _ptr(vel), _ptr(acc), pos.shape[0], float(box), int(K), int(R),
                              float(eps), _ptr(dt), ctypes.byref(prm) if prm is not None else None, _ptr(ws),
                              ws.numel() * ws.element_size(), _stream(stream)),
           "nf_kdk_step")


def nf_multipoles(pos: torch.Tensor, box: float, K: int, p: int, M: torch.Tensor, ws: torch.Tensor,
                  stream=None) -> None:
    _check(load().nf_multipoles(_ptr(pos), pos.shape[0], float(box), int(K), int(p), _ptr(M), _ptr(ws),
                                ws.numel() * ws.element_size(), _stream(stream)),
           "nf_multipoles")


def nf_derivatives_bytes(K: int, p: int) -> int:
    return int(load().nf_derivatives_bytes(int(K), int(p)))


def nf_far_workspace_bytes(N: int, K: int, p: int) -> int:
    return int(load().nf_far_workspace_bytes(int(N), int(K), int(p)))


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


def nf_derivatives(K: int, R: int, p: int, box: float, derivs: torch.Tensor, ws: torch.Tensor,
                   stream=None) -> None:
    _check(load().nf_derivatives(int(K), int(R), int(p), float(box), _ptr(derivs), _nbytes(derivs), _ptr(ws),
                                 _nbytes(ws), _stream(stream)), "nf_derivatives")


def nf_far_forces(pos: torch.Tensor, box: float, K: int, R: int, p: int, derivs: torch.Tensor,
                  acc_far: Optional[torch.Tensor], acc_add: Optional[torch.Tensor],
                  taylors: Optional[torch.Tensor], ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_far_forces(_ptr(pos), pos.shape[0], float(box), int(K), int(R), int(p), _ptr(derivs),
                                _nbytes(derivs), _ptr(acc_far), _ptr(acc_add), _ptr(taylors), _ptr(ws),
                                _nbytes(ws), _stream(stream)), "nf_far_forces")


def nf_kdk_step_far(pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, box: float, K: int, R: int,
                    eps: float, p: int, derivs: torch.Tensor, dt: torch.Tensor, prm, ws: torch.Tensor,
                    ws_far: torch.Tensor, stream=None) -> None:
    _check(load().nf_kdk_step_far(_ptr(pos), _ptr(vel), _ptr(acc), pos.shape[0], float(box), int(K), int(R),
                                  float(eps), int(p), _ptr(derivs), _nbytes(derivs), _ptr(dt),
                                  None if prm is None else ctypes.byref(prm), _ptr(ws), _nbytes(ws),
                                  _ptr(ws_far), _nbytes(ws_far), _stream(stream)), "nf_kdk_step_far")


def nf_forces_total(pos: torch.Tensor, box: float, K: int, R: int, eps: float, p: int, derivs: torch.Tensor,
                    acc: torch.Tensor, ws: torch.Tensor, ws_far: torch.Tensor, stream=None) -> None:
    _check(load().nf_forces_total(_ptr(pos), pos.shape[0], float(box), int(K), int(R), float(eps), int(p),
                                  _ptr(derivs), _nbytes(derivs), _ptr(acc), _ptr(ws), _nbytes(ws), _ptr(ws_far),
                                  _nbytes(ws_far), _stream(stream)), "nf_forces_total")


NF_FAR_FP64, NF_FAR_DOUBLE_FLOAT = 0, 1


def nf_far_set_arith(mode: int) -> None:
    _check(load().nf_far_set_arith(int(mode)), "nf_far_set_arith")


def nf_far_get_arith() -> int:
    return int(load().nf_far_get_arith())


def nf_far_release() -> None:
    _check(load().nf_far_release(), "nf_far_release")


NF_DENS_AUTO, NF_DENS_FUSED, NF_DENS_DEFERRED = 0, 1, 2


def nf_set_density_mode(mode: int) -> None:
    _check(load().nf_set_density_mode(int(mode)), "nf_set_density_mode")


def nf_get_density_mode() -> int:
    return int(load().nf_get_density_mode())


def nf_set_debug(on: bool) -> None:
    _check(load().nf_set_debug(1 if on else 0), "nf_set_debug")


def nf_debug_check(ws: torch.Tensor, stream=None) -> None:
    _check(load().nf_debug_check(_ptr(ws), _stream(stream)), "nf_debug_check")
