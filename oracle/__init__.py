"""FP64 CPU oracle for the near-field force: TEST INFRASTRUCTURE ONLY.

The oracle is the plain, slow reference the CUDA path is checked against
(binning, near-field accelerations, their adjoint, and a local energy for
finite differences).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The product path never calls
it and shares no code with it.

The arithmetic lives in ``nf_oracle.c`` (plain C, FP64, OpenMP over sinks),
compiled here with ``-O2 -ffp-contract=off`` so no FMA contraction changes the
binning's rounding.  Each function below cites what it follows in the paper
(Garrison et al., "The Abacus Cosmological N-body Code"):

* :func:`bin_particles` - cell-centred FP32 offsets on the K^3 grid
  (Sec. "Force Accuracy" overview; Sec. "Two-Stage Execution").
* :func:`forces` - near-field sum over the (2R+1)^3 neighbour cells with the
  spline softening of Eq. (spline), eps_s = 2.16 eps_p (Sec. "Force Softening";
  Sec. "GPU Near-Field Computation").
* :func:`adjoint` - gradient of L = sum_i g_i . a_i (not in the paper; the
  derivative of the sum above).
* :class:`Grid` - the same two sums on a particle set binned once, for
  several sink samples of one large set.
* :func:`local_energy` - the part of L that depends on one particle, for
  finite differences with frozen cell assignment.
* :func:`timestep` - the global time step of Eq. (timestep), Sec. "Time
  Stepping": per-cell v_rms / a_max (v_rms without subtracting the cell's
  mean velocity), the most conservative cell, guarded by the global ratio
  and limited by the Hubble term.
* :func:`kdk_step` - one Kick-Drift-Kick leapfrog step (Sec. "Time
  Stepping") with the near-field accelerations of :func:`forces`.
* :func:`multipoles` - cell multipoles in the complete basis, Eq. (multipoles)
  (Sec. "Computation of the Cell Multipoles"), about the cell centres.
* :func:`derivatives`, :func:`taylors_fft`, :func:`taylor_forces`,
  :func:`far_field` - the far field of Sec. "Far-field Computation": the
  derivatives tensor (all periodic images by Ewald's split, minus the image
  the near field computes), the Taylors as the convolution of derivatives and
  multipoles (by FFT; :func:`convolve_direct` is the plain cyclic sum), and
  the acceleration from the Taylors.  The arithmetic is in ``nf_oracle_far.c``.
* :func:`ewald_forces` - plain Ewald summation over every pair, the reference
  the paper's Sec. "Force Accuracy" compares the total force against.
* :func:`density` - the apodized top-hat density estimate the paper's kernel
  accumulates as a 4th component, sum over near-field j with r < b of
  (1 - r^2/b^2) (Sec. "Force Kernel").

Every function has at least one pin in ``tests/test_oracle_pins.py`` against
closed forms, brute force, symmetry or the paper's printed values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nf_oracle.c")
_SRC_FAR = os.path.join(_HERE, "nf_oracle_far.c")
_LIB_PATH = os.path.join(_HERE, "_nf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp -ffp-contract=off)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_FAR)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=c11", "-o", tmp, _SRC, _SRC_FAR, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_bin.restype = i64
    lib.oracle_bin.argtypes = [P, i64, f64, i32, P, P, P, P]
    lib.oracle_forces.restype = i32
    lib.oracle_forces.argtypes = [P, i64, f64, i32, i32, f64, P, i64, P, i32]
    lib.oracle_adjoint.restype = i32
    lib.oracle_adjoint.argtypes = [P, P, i64, f64, i32, i32, f64, P, i64, P, i32]
    lib.oracle_local_energy.restype = i32
    lib.oracle_local_energy.argtypes = [P, P, i64, f64, i32, i32, f64, P, i64, P, P]
    lib.oracle_density.restype = i32
    lib.oracle_density.argtypes = [P, i64, f64, i32, i32, f64, P, i64, P, i32]
    lib.oracle_multipoles.restype = i32
    lib.oracle_multipoles.argtypes = [P, i64, f64, i32, i32, P]
    lib.oracle_multipole_terms.restype = i64
    lib.oracle_multipole_terms.argtypes = [i32]
    lib.oracle_wrapped_positions.restype = i32
    lib.oracle_wrapped_positions.argtypes = [P, i64, f64, i32, P]
    lib.oracle_num_threads.restype = i32
    lib.oracle_num_threads.argtypes = []
    lib.oracle_derivatives.restype = i32
    lib.oracle_derivatives.argtypes = [i32, i32, i32, f64, f64, i32, i32, P]
    lib.oracle_coulomb_derivatives.restype = None
    lib.oracle_coulomb_derivatives.argtypes = [i32, f64, f64, f64, P]
    lib.oracle_convolve_direct.restype = i32
    lib.oracle_convolve_direct.argtypes = [i32, i32, P, P, P]
    lib.oracle_taylor_forces.restype = i32
    lib.oracle_taylor_forces.argtypes = [P, i64, f64, i32, i32, P, P]
    lib.oracle_ewald_forces.restype = i32
    lib.oracle_ewald_forces.argtypes = [P, i64, f64, f64, i32, i32, P, i64, P]
    lib.oracle_grid_new.restype = P
    lib.oracle_grid_new.argtypes = [P, i64, f64, i32, i32, f64]
    lib.oracle_grid_delete.restype = None
    lib.oracle_grid_delete.argtypes = [P]
    lib.oracle_grid_binning.restype = None
    lib.oracle_grid_binning.argtypes = [P, P, P]
    lib.oracle_grid_forces.restype = None
    lib.oracle_grid_forces.argtypes = [P, P, i64, P, i32]
    lib.oracle_grid_adjoint.restype = None
    lib.oracle_grid_adjoint.argtypes = [P, P, P, i64, P, i32]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pos(pos) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pos, dtype=np.float32))
    assert a.ndim == 2 and a.shape[1] == 3
    return a


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def bin_particles(pos, box: float, K: int):
    """Stable binning: returns (cell_offsets int32[K^3+1], rel float32[N,4], perm int32[N]).

    rel[:, :3] are FP32 offsets from the cell centre in cell units; rel[:, 3]
    holds the bits of the original index.  Raises on non-finite input.
    """
    pos = _pos(pos)
    N = pos.shape[0]
    off = np.zeros(K ** 3 + 1, np.int32)
    rel = np.zeros((max(N, 1), 4), np.float32)
    perm = np.zeros(max(N, 1), np.int32)
    bad = _load().oracle_bin(_p(pos), N, float(box), int(K), _p(off), _p(rel), _p(perm), None)
    if bad:
        raise ValueError(f"{bad} non-finite coordinates")
    return off, rel[:N], perm[:N]


def cell_of(pos, box: float, K: int) -> np.ndarray:
    """Linear cell index (cx*K + cy)*K + cz of every particle, input order."""
    pos = _pos(pos)
    N = pos.shape[0]
    off = np.zeros(K ** 3 + 1, np.int32)
    rel = np.zeros((max(N, 1), 4), np.float32)
    perm = np.zeros(max(N, 1), np.int32)
    cid = np.zeros(max(N, 1), np.int32)
    bad = _load().oracle_bin(_p(pos), N, float(box), int(K), _p(off), _p(rel), _p(perm), _p(cid))
    if bad:
        raise ValueError(f"{bad} non-finite coordinates")
    return cid[:N]


def forces(pos, box: float, K: int, R: int, eps: float,
           sinks: Optional[np.ndarray] = None, threads: int = 0) -> np.ndarray:
    """Near-field accelerations in FP64, [N, 3] (or [len(sinks), 3]).

    eps is the Plummer-equivalent softening in box units; mass 1/N, G = 1.
    """
    pos = _pos(pos)
    N = pos.shape[0]
    s = None if sinks is None else np.ascontiguousarray(np.asarray(sinks, np.int64))
    n = N if s is None else s.shape[0]
    out = np.zeros((max(n, 1), 3), np.float64)
    rc = _load().oracle_forces(_p(pos), N, float(box), int(K), int(R), float(eps),
                               None if s is None else _p(s), n, _p(out), int(threads))
    if rc:
        raise ValueError("non-finite coordinates")
    return out[:n]


def adjoint(pos, g, box: float, K: int, R: int, eps: float,
            sinks: Optional[np.ndarray] = None, threads: int = 0) -> np.ndarray:
    """dL/dx for L = sum_i g_i . a_i, FP64 [N, 3] (or at the listed sinks)."""
    pos = _pos(pos)
    N = pos.shape[0]
    gg = np.ascontiguousarray(np.asarray(g, np.float64).reshape(N, 3))
    s = None if sinks is None else np.ascontiguousarray(np.asarray(sinks, np.int64))
    n = N if s is None else s.shape[0]
    out = np.zeros((max(n, 1), 3), np.float64)
    rc = _load().oracle_adjoint(_p(pos), _p(gg), N, float(box), int(K), int(R), float(eps),
                                None if s is None else _p(s), n, _p(out), int(threads))
    if rc:
        raise ValueError("non-finite coordinates")
    return out[:n]


class Grid:
    """One particle set binned once for several sink samples.

    ``Grid(pos, box, K, R, eps).forces(sinks)`` equals ``forces(pos, box, K,
    R, eps, sinks=sinks)`` exactly (the same set-up and the same sums), and
    likewise :meth:`adjoint`; the binning of all particles, which those
    functions repeat on every call, is done once here.
    """

    def __init__(self, pos, box: float, K: int, R: int, eps: float):
        self.pos = _pos(pos)
        self.N = self.pos.shape[0]
        self.K = int(K)
        lib = _load()
        self._h = lib.oracle_grid_new(_p(self.pos), self.N, float(box), self.K, int(R), float(eps))
        if not self._h:
            raise ValueError("non-finite coordinates (or out of memory)")

    def binning(self):
        """(cell_offsets int32[K^3+1], perm int32[N]) of the stable binning."""
        off = np.zeros(self.K ** 3 + 1, np.int32)
        perm = np.zeros(max(self.N, 1), np.int32)
        _load().oracle_grid_binning(self._h, _p(off), _p(perm))
        return off, perm[:self.N]

    def forces(self, sinks: np.ndarray, threads: int = 0) -> np.ndarray:
        s = np.ascontiguousarray(np.asarray(sinks, np.int64))
        out = np.zeros((max(s.shape[0], 1), 3), np.float64)
        _load().oracle_grid_forces(self._h, _p(s), s.shape[0], _p(out), int(threads))
        return out[:s.shape[0]]

    def adjoint(self, g, sinks: np.ndarray, threads: int = 0) -> np.ndarray:
        gg = np.ascontiguousarray(np.asarray(g, np.float64).reshape(self.N, 3))
        s = np.ascontiguousarray(np.asarray(sinks, np.int64))
        out = np.zeros((max(s.shape[0], 1), 3), np.float64)
        _load().oracle_grid_adjoint(self._h, _p(gg), _p(s), s.shape[0], _p(out), int(threads))
        return out[:s.shape[0]]

    def close(self):
        if getattr(self, "_h", None):
            _load().oracle_grid_delete(self._h)
            self._h = None

    def __del__(self):
        self.close()


def multipole_terms(p: int) -> int:
    return int(_load().oracle_multipole_terms(int(p)))


def multipole_index(p: int):
    """(a, b, c) of every complete-basis term, in the order of the output."""
    return [(a, b, c) for a in range(p + 1) for b in range(p + 1 - a) for c in range(p + 1 - a - b)]


def multipoles(pos, box: float, K: int, p: int) -> np.ndarray:
    """M[cell, term] = sum over the cell's particles of x^a y^b z^c, FP64, with
    (x, y, z) the displacement from the cell centre in box units (the stored
    FP32 cell-centred offset times the cell width); terms in the order of
    multipole_index(p)."""
    pos = _pos(pos)
    N = pos.shape[0]
    nt = multipole_terms(p)
    M = np.zeros((K ** 3, nt), np.float64)
    if _load().oracle_multipoles(_p(pos), N, float(box), int(K), int(p), _p(M)):
        raise ValueError("non-finite coordinates")
    return M


def density(pos, box: float, K: int, R: int, b: float,
            sinks: Optional[np.ndarray] = None, threads: int = 0) -> np.ndarray:
    """Top-hat density estimate, FP64 [N] (or [len(sinks)]): sum over the
    near-field neighbours j (self included) with r_ij < b of 1 - r_ij^2/b^2."""
    pos = _pos(pos)
    N = pos.shape[0]
    s = None if sinks is None else np.ascontiguousarray(np.asarray(sinks, np.int64))
    n = N if s is None else s.shape[0]
    out = np.zeros(max(n, 1), np.float64)
    rc = _load().oracle_density(_p(pos), N, float(box), int(K), int(R), float(b),
                                None if s is None else _p(s), n, _p(out), int(threads))
    if rc:
        raise ValueError("non-finite coordinates")
    return out[:n]


def timestep(vel, acc, cell, eta_acc: float, eta_h: float = 0.0, hubble: float = 0.0) -> float:
    """dt = min(eta_H / H, eta_acc * max(min_c v_rms,c / a_max,c, v_rms / a_max)) in FP64.

    Eq. (timestep) written for dt with a = 1 (dt = da / (a H)); cell[i] is the
    cell of particle i.  Cells whose largest acceleration is zero are skipped;
    with H = 0 there is no Hubble limit.  Returns +inf if nothing limits dt.
    """
    v2 = (np.asarray(vel, np.float64) ** 2).sum(axis=1)
    a = np.sqrt((np.asarray(acc, np.float64) ** 2).sum(axis=1))
    cell = np.asarray(cell)
    best = np.inf
    for c in np.unique(cell):
        sel = cell == c
        amax = a[sel].max()
        if amax > 0.0:
            best = min(best, np.sqrt(v2[sel].mean()) / amax)
    amax_g = a.max()
    glob = np.sqrt(v2.mean()) / amax_g if amax_g > 0.0 else np.inf
    dt = eta_acc * max(best, glob) if np.isfinite(max(best, glob)) else np.inf
    if hubble > 0.0:
        dt = min(dt, eta_h / hubble)
    return float(dt)


def kdk_step(pos, vel, acc, dt: float, box: float, K: int, R: int, eps: float,
             far_order: Optional[int] = None, D: Optional[np.ndarray] = None):
    """One leapfrog step: v += a dt/2; x += v dt (wrapped into [0, box)); a = F(x);
    v += a dt/2.  State stored as the API stores it (FP32 positions and
    velocities); arithmetic in FP64.  F is the near field, plus the far field
    of order far_order (derivatives D, computed when not given) when far_order
    is set.  Returns (pos, vel, acc_FP64)."""
    pos = np.asarray(pos, np.float32)
    v = np.asarray(vel, np.float32).astype(np.float64)
    a = np.asarray(acc, np.float64)
    v_half = (v + 0.5 * dt * a).astype(np.float32)
    x = pos.astype(np.float64) + dt * v_half.astype(np.float64)
    x = np.mod(x, box).astype(np.float32)
    x[x >= np.float32(box)] = np.float32(0.0)
    a_new = forces(x, box, K, R, eps)
    if far_order is not None:
        a_new = a_new + far_field(x, box, K, R, far_order, D=D)
    v_new = (v_half.astype(np.float64) + 0.5 * dt * a_new).astype(np.float32)
    return x, v_new, a_new


def local_energy(pos, g, box: float, K: int, R: int, eps: float,
                 ks: np.ndarray, xk: np.ndarray) -> np.ndarray:
    """L_k with particle ks[q] moved to the FP64 position xk[q] (cells frozen)."""
    pos = _pos(pos)
    N = pos.shape[0]
    gg = np.ascontiguousarray(np.asarray(g, np.float64).reshape(N, 3))
    ks = np.ascontiguousarray(np.asarray(ks, np.int64))
    xk = np.ascontiguousarray(np.asarray(xk, np.float64).reshape(ks.shape[0], 3))
    out = np.zeros(max(ks.shape[0], 1), np.float64)
    rc = _load().oracle_local_energy(_p(pos), _p(gg), N, float(box), int(K), int(R), float(eps),
                                     _p(ks), ks.shape[0], _p(xk), _p(out))
    if rc:
        raise ValueError("non-finite coordinates")
    return out[:ks.shape[0]]


def wrapped_positions(pos, box: float, K: int) -> np.ndarray:
    """FP64 positions moved into [0, box) by whole boxes, as the force sums use them."""
    pos = _pos(pos)
    out = np.zeros((max(pos.shape[0], 1), 3), np.float64)
    if _load().oracle_wrapped_positions(_p(pos), pos.shape[0], float(box), int(K), _p(out)):
        raise ValueError("non-finite coordinates")
    return out[:pos.shape[0]]


def fd_gradient(pos, g, box: float, K: int, R: int, eps: float, ks: np.ndarray,
                h: float = 1e-6) -> np.ndarray:
    """Central finite differences of the local energy, step h (box units), [len(ks), 3]."""
    xw = wrapped_positions(pos, box, K)
    ks = np.asarray(ks, np.int64)
    grad = np.zeros((ks.shape[0], 3))
    for d in range(3):
        xp = xw[ks].copy()
        xm = xw[ks].copy()
        xp[:, d] += h
        xm[:, d] -= h
        lp = local_energy(pos, g, box, K, R, eps, ks, xp)
        lm = local_energy(pos, g, box, K, R, eps, ks, xm)
        grad[:, d] = (lp - lm) / (2.0 * h)
    return grad


def frac_error(a: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """|a_i - ref_i|_2 / |ref_i|_2 per particle (no floor)."""
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


# ---------------------------------------------------------------------------
# far field (Sec. "Far-field Computation") and the Ewald reference
# ---------------------------------------------------------------------------

EWALD_ALPHA_L = 3.5   # alpha * box of the default Ewald split
EWALD_NIMG = 2        # real-space images n in [-2, 2]^3
EWALD_HMAX = 9        # reciprocal vectors h in [-9, 9]^3


def derivatives(K: int, R: int, p: int, box: float = 1.0, alpha: Optional[float] = None,
                nimg: int = EWALD_NIMG, hmax: int = EWALD_HMAX) -> np.ndarray:
    """Derivatives tensor D[g, term] (g = (gx*K + gy)*K + gz the sink-minus-source
    cell offset mod K; terms in multipole_index(p) order): Cartesian derivatives
    of the periodic unit-mass potential over all images, minus the near-field
    image, at the cell-centre separation.  alpha defaults to 3.5 / box."""
    a = EWALD_ALPHA_L / box if alpha is None else float(alpha)
    D = np.zeros((K ** 3, multipole_terms(p)), np.float64)
    _load().oracle_derivatives(int(K), int(R), int(p), float(box), a, int(nimg), int(hmax), _p(D))
    return D


def coulomb_derivatives(p: int, r) -> np.ndarray:
    """Cartesian derivatives of 1/|r| at r != 0, every term of order <= p."""
    out = np.zeros(multipole_terms(p), np.float64)
    _load().oracle_coulomb_derivatives(int(p), float(r[0]), float(r[1]), float(r[2]), _p(out))
    return out


def taylor_coefficients(p: int):
    """(n, k, n+k) term indices and (-1)^|k| / (n! k!) for every |n| + |k| <= p."""
    from math import factorial
    idx = multipole_index(p)
    where = {t: q for q, t in enumerate(idx)}
    out = []
    for qn, n in enumerate(idx):
        for qk, k in enumerate(idx):
            if sum(n) + sum(k) > p:
                continue
            j = (n[0] + k[0], n[1] + k[1], n[2] + k[2])
            coef = (-1.0) ** sum(k) / float(factorial(n[0]) * factorial(n[1]) * factorial(n[2]) *
                                          factorial(k[0]) * factorial(k[1]) * factorial(k[2]))
            out.append((qn, qk, where[j], coef))
    return out


def convolve_direct(K: int, p: int, D: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Taylors T[cell, term] by the plain cyclic sum over every (sink, source) cell pair."""
    T = np.zeros((K ** 3, multipole_terms(p)), np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    _load().oracle_convolve_direct(int(K), int(p), _p(D), _p(M), _p(T))
    return T


def taylors_fft(K: int, p: int, D: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Taylors T[cell, term]: the same convolution through numpy's 3-D FFT."""
    nt = multipole_terms(p)
    Dh = np.fft.fftn(D.reshape(K, K, K, nt), axes=(0, 1, 2))
    Mh = np.fft.fftn(M.reshape(K, K, K, nt), axes=(0, 1, 2))
    Th = np.zeros_like(Dh)
    for qn, qk, qj, coef in taylor_coefficients(p):
        Th[..., qn] += coef * Dh[..., qj] * Mh[..., qk]
    return np.fft.ifftn(Th, axes=(0, 1, 2)).real.reshape(K ** 3, nt)


def taylor_forces(pos, box: float, K: int, p: int, T: np.ndarray) -> np.ndarray:
    """sum_n T^n grad(x^n) at every particle (unit masses), input order."""
    pos = _pos(pos)
    out = np.zeros((pos.shape[0], 3), np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    if _load().oracle_taylor_forces(_p(pos), pos.shape[0], float(box), int(K), int(p), _p(T), _p(out)):
        raise ValueError("non-finite coordinates")
    return out


def far_field(pos, box: float, K: int, R: int, p: int, D: Optional[np.ndarray] = None,
              return_taylors: bool = False):
    """Far-field accelerations (m = 1/N, G = 1): multipoles, convolution with the
    derivatives tensor, Taylor evaluation."""
    pos = _pos(pos)
    N = pos.shape[0]
    if D is None:
        D = derivatives(K, R, p, box)
    M = multipoles(pos, box, K, p)
    T = taylors_fft(K, p, D, M)
    a = taylor_forces(pos, box, K, p, T) / N
    return (a, T) if return_taylors else a


def ewald_forces(pos, box: float, sinks: Optional[np.ndarray] = None, alpha: Optional[float] = None,
                 nimg: int = 1, hmax: int = EWALD_HMAX) -> np.ndarray:
    """Plain Ewald accelerations (m = 1/N, G = 1, unsoftened) on the sinks (all by default).

    Pair separations are first reduced to the minimum image, so with
    alpha * box = 3.5 the images n in [-1, 1]^3 leave out only terms below
    erfc(5.25) ~ 1e-13 of a unit pair force."""
    pos = _pos(pos)
    N = pos.shape[0]
    a = EWALD_ALPHA_L / box if alpha is None else float(alpha)
    s = None if sinks is None else np.ascontiguousarray(sinks, dtype=np.int64)
    n = N if s is None else len(s)
    out = np.zeros((n, 3), np.float64)
    if _load().oracle_ewald_forces(_p(pos), N, float(box), a, int(nimg), int(hmax),
                                   None if s is None else _p(s), n, _p(out)):
        raise ValueError("non-finite coordinates")
    return out / N
