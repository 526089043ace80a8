"""The benchmark's multiply-add throughput probe (libnf_probe.so).

A measurement aid, not part of libnf's C ABI: it gives the measured FP32 and
FP64 multiply-add rates the benchmark reports beside the derived peaks of its
rooflines.  One launch of 4 blocks of 256 threads per SM; every thread runs 8
independent multiply-add chains for iters x 16 trips as scalar fma.rn.f32
(mode 0), packed fma.rn.f32x2 (mode 1) or fma.rn.f64 (mode 2).
"""
from __future__ import annotations

import ctypes

import torch

from . import _build

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_probe())
        lib.nfp_fma_probe_sink_floats.restype = ctypes.c_size_t
        lib.nfp_fma_probe_sink_floats.argtypes = []
        lib.nfp_fma_probe.restype = ctypes.c_int
        lib.nfp_fma_probe.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p]
        _lib = lib
    return _lib


def sink_floats() -> int:
    """Values the sink buffer must hold (one per thread of the launch)."""
    return int(load().nfp_fma_probe_sink_floats())


def fma_probe(sink: torch.Tensor, iters: int, mode, stream=None) -> float:
    """Launches the probe on `stream` (default: the current stream) and returns
    the floating-point operations of the launch (2 per multiply-add and lane).
    mode: 0 f32, 1 f32x2 (True also means packed), 2 f64."""
    if sink.dtype != torch.float32 or not sink.is_cuda or sink.numel() < sink_floats():
        raise ValueError("sink must be a CUDA float32 tensor of sink_floats() values")
    s = stream if stream is not None else torch.cuda.current_stream(sink.device)
    flop = ctypes.c_double(0.0)
    rc = load().nfp_fma_probe(ctypes.c_void_p(sink.data_ptr()), int(iters), int(mode), ctypes.byref(flop),
                              ctypes.c_void_p(s.cuda_stream))
    if rc == 1:
        raise ValueError(f"fma_probe: bad argument (iters {iters}, mode {mode})")
    if rc:
        raise RuntimeError(f"fma_probe: CUDA error {rc - 2}")
    return flop.value
