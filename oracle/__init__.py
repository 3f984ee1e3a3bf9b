"""FP64 CPU oracle for Richardson-Lucy deconvolution (Welk & Erler).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports it, and
this package imports nothing from the product path.

The arithmetic lives in ``rl_oracle.c`` (plain C, double precision, direct
summation over the PSF support; Eq. 3 of Sec. 2, the boundary rules of Sec. 2,
Eq. 4-5 of Sec. 4).  This module only marshals numpy arrays through ctypes and
compiles the C file with gcc on first use (``build()``).

PSF objects are :class:`Psf`: a dense ``(kh, kw)`` float64 tap array whose entry
``[j, i]`` sits at offset ``(i - ax, j - ay)`` from the origin.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rl_oracle.c")
_LIB = os.path.join(_HERE, "_rl_oracle.so")
_lock = threading.Lock()
_lib = None

MIRROR = 0
CLAMP = 1
PADFLIP = 0
TRANSPOSE = 1

_BOUNDARY = {"mirror": MIRROR, "clamp": CLAMP, MIRROR: MIRROR, CLAMP: CLAMP}
_ADJOINT = {"padflip": PADFLIP, "transpose": TRANSPOSE, PADFLIP: PADFLIP,
            TRANSPOSE: TRANSPOSE}


def build(force: bool = False) -> str:
    """Compile ``rl_oracle.c`` into ``_rl_oracle.so`` (gcc, OpenMP, no FMA
    contraction so that x86 and Arm hosts round identically)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d = ctypes.POINTER(ctypes.c_double)
    i = ctypes.c_int
    lib.orc_map.restype = ctypes.c_long
    lib.orc_map.argtypes = [ctypes.c_long, ctypes.c_long, i]
    lib.orc_psf_normalize.restype = i
    lib.orc_psf_normalize.argtypes = [d, i]
    lib.orc_psf_motion.restype = i
    lib.orc_psf_motion.argtypes = [i, i, d] + [ctypes.POINTER(i)] * 4
    lib.orc_psf_disc.restype = i
    lib.orc_psf_disc.argtypes = [i, d] + [ctypes.POINTER(i)] * 4
    conv_args = [d, d, i, i, d, i, i, i, i, i]
    for name in ("orc_conv", "orc_conv_padflip", "orc_conv_transpose"):
        getattr(lib, name).restype = None
        getattr(lib, name).argtypes = conv_args
    lib.orc_rl.restype = i
    lib.orc_rl.argtypes = [d, d, d, i, i, d, i, i, i, i, i, i, i, i,
                           ctypes.c_double, i, i, i,
                           ctypes.POINTER(ctypes.c_uint8),
                           ctypes.POINTER(ctypes.c_longlong)]
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclasses.dataclass(frozen=True)
class Psf:
    """Dense PSF: ``taps[j, i]`` at offset ``(i - ax, j - ay)``."""
    taps: np.ndarray
    ax: int
    ay: int

    @property
    def kh(self) -> int:
        return self.taps.shape[0]

    @property
    def kw(self) -> int:
        return self.taps.shape[1]


def psf_motion(length: int, axis: int = 0) -> Psf:
    """Uniform linear motion blur along x (axis 0) or y (axis 1), Sec. 3,
    Fig. 1a; anchor at index length//2."""
    lib = _load()
    h = np.zeros(length, np.float64)
    kw, kh, ax, ay = (ctypes.c_int() for _ in range(4))
    if lib.orc_psf_motion(length, axis, _dptr(h), kw, kh, ax, ay) != 0:
        raise ValueError("bad motion PSF")
    return Psf(h.reshape(kh.value, kw.value), ax.value, ay.value)


def psf_disc(radius: int) -> Psf:
    """Pillbox of radius r by pixel-centre inclusion, Sec. 3 "Defocus blur"."""
    lib = _load()
    n = 2 * radius + 1
    h = np.zeros(n * n, np.float64)
    kw, kh, ax, ay = (ctypes.c_int() for _ in range(4))
    if lib.orc_psf_disc(radius, _dptr(h), kw, kh, ax, ay) < 0:
        raise ValueError("bad disc PSF")
    return Psf(h.reshape(n, n), ax.value, ay.value)


def psf_dense(taps, ax: int | None = None, ay: int | None = None) -> Psf:
    """Dense taps normalised to unit sum; the anchor defaults to the centre
    ``(kw//2, kh//2)``.  Raises ValueError on negative / non-finite taps or a
    non-positive sum."""
    lib = _load()
    t = _f64(np.atleast_2d(taps)).copy()
    if lib.orc_psf_normalize(_dptr(t.reshape(-1)), t.size) != 0:
        raise ValueError("PSF taps must be finite, >= 0, with positive sum")
    kh, kw = t.shape
    return Psf(t, kw // 2 if ax is None else ax, kh // 2 if ay is None else ay)


def bmap(e: int, n: int, boundary="mirror") -> int:
    return int(_load().orc_map(e, n, _BOUNDARY[boundary]))


def _conv_call(name, img, psf: Psf, boundary):
    lib = _load()
    a = _f64(img)
    H, W = a.shape
    out = np.empty_like(a)
    taps = _f64(psf.taps)
    getattr(lib, name)(_dptr(a), _dptr(out), W, H, _dptr(taps), psf.kw,
                       psf.kh, psf.ax, psf.ay, _BOUNDARY[boundary])
    return out


def conv(u, psf: Psf, boundary="mirror") -> np.ndarray:
    """Forward operator A: v = h (x) u with the given boundary continuation."""
    return _conv_call("orc_conv", u, psf, boundary)


def conv_adjoint(q, psf: Psf, boundary="mirror", adjoint="padflip"):
    """Adjoint operator: ``padflip`` = convolution with the reflected PSF under
    the same boundary continuation (Eq. 3 read literally); ``transpose`` = the
    exact matrix transpose A^T."""
    name = ("orc_conv_transpose" if _ADJOINT[adjoint] == TRANSPOSE
            else "orc_conv_padflip")
    return _conv_call(name, q, psf, boundary)


@dataclasses.dataclass
class RLResult:
    u: np.ndarray
    active_pixel_iterations: int
    mask_trace: np.ndarray | None


def rl(f, psf: Psf, iterations: int, u0=None, boundary="mirror",
       adjoint="padflip", threshold: float | None = None,
       relative: bool = True, reset_period: int = 10,
       update_period: int = 1, want_mask: bool = False) -> RLResult:
    """Richardson-Lucy (Eq. 3) with optional selective convolution (Eq. 4-5).

    ``threshold=None`` runs plain RL.  ``update_period`` is 1 (mask checked
    every iteration, Sec. 4) or ``reset_period`` (mask recomputed only on the
    full iterations).  ``want_mask`` returns the per-iteration "used" masks
    as a ``(K, H, W)`` uint8 array.
    """
    lib = _load()
    fa = _f64(f)
    H, W = fa.shape
    u = np.empty_like(fa)
    u0a = None if u0 is None else _f64(u0)
    taps = _f64(psf.taps)
    trace = (np.zeros((iterations, H, W), np.uint8)
             if want_mask and iterations > 0 else None)
    act = ctypes.c_longlong(0)
    thin = threshold is not None
    rc = lib.orc_rl(_dptr(fa), None if u0a is None else _dptr(u0a), _dptr(u),
                    W, H, _dptr(taps), psf.kw, psf.kh, psf.ax, psf.ay,
                    _BOUNDARY[boundary], _ADJOINT[adjoint], int(iterations),
                    int(thin), float(threshold or 0.0), int(bool(relative)),
                    int(reset_period), int(update_period),
                    None if trace is None else
                    trace.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                    ctypes.byref(act))
    if rc != 0:
        raise ValueError("oracle rl: bad arguments")
    return RLResult(u, int(act.value), trace)


def snr_db(u, g) -> float:
    """SNR of u against g: 10 log10(Var(g) / MSE(u, g)) (the paper does not
    define its SNR; this is the reading used throughout)."""
    g = _f64(g)
    mse = float(np.mean((_f64(u) - g) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(float(np.var(g)) / mse)


def psnr_db(u, g) -> float:
    """PSNR with peak = max(g)."""
    g = _f64(g)
    mse = float(np.mean((_f64(u) - g) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(float(g.max()) ** 2 / mse)


def rel_linf(a, b) -> float:
    """Relative L-infinity error max|a - b| / max|b|."""
    b = _f64(b)
    return float(np.max(np.abs(_f64(a) - b)) / max(np.max(np.abs(b)), 1e-300))
