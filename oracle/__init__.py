"""FP64 CPU oracle of STORM-GPA (arXiv 2604.16590, Sec. III-C).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and it imports nothing of the
library: the two share no code.

The arithmetic lives in ``gpa_oracle.c`` (plain FP64 loops, OpenMP over
independent (batch*head, tile) units); this module compiles it with gcc on
first use and wraps it with numpy.  ``brute.py`` holds an independent dense
brute force used to pin it.

Geometry is passed as ``(B, nh, d, T, Y, X, core, halo)``; tensors are
``[B, nh, N, d]`` float64 with token i = (t*Y + y)*X + x.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgpa_oracle.so")
_lock = threading.Lock()
_lib = None

WINDOWS = {"hann": 0, "flat": 1}


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/libgpa_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            I64 = ctypes.c_int64
            lib.gpa_num_tiles.argtypes = [P]
            lib.gpa_num_tiles.restype = I
            lib.gpa_tile_rows.argtypes = [P, I]
            lib.gpa_tile_rows.restype = I
            lib.gpa_window_1d.argtypes = [I, I]
            lib.gpa_window_1d.restype = D
            lib.gpa_oracle_threads.restype = I
            lib.gpa_forward.argtypes = [P, I, D, P, P, P, P]
            lib.gpa_backward.argtypes = [P, I, D, P, P, P, P, P, P, P]
            lib.gpa_rows.argtypes = [P, I, D, P, P, P, P, I64, P, P, P]
            lib.gpa_key_rows.argtypes = [P, I, D, P, P, P, P, I64, P, P, P]
            lib.gpa_unit_fwd_bwd.argtypes = [P, I, D, P, P, P, P, I, I, I, I]
            _lib = lib
    return _lib


def _geom(B, nh, d, T, Y, X, core, halo) -> np.ndarray:
    g = np.array([B, nh, d, T, Y, X, *core, *halo], dtype=np.int32)
    assert g.shape == (12,)
    return g


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Geometry:
    """Token grid, tile spec and head layout of one GPA call."""

    def __init__(self, B, nh, d, T, Y, X, core, halo, window="hann", scale=None):
        self.B, self.nh, self.d = int(B), int(nh), int(d)
        self.T, self.Y, self.X = int(T), int(Y), int(X)
        self.core = tuple(int(c) for c in core)
        self.halo = tuple(int(h) for h in halo)
        self.window = window
        self.scale = float(scale) if scale is not None else 1.0 / np.sqrt(self.d)
        self.g = _geom(self.B, self.nh, self.d, self.T, self.Y, self.X, self.core, self.halo)

    @property
    def N(self) -> int:
        return self.T * self.Y * self.X

    @property
    def shape(self):
        return (self.B, self.nh, self.N, self.d)

    def num_tiles(self) -> int:
        return _load().gpa_num_tiles(_ptr(self.g))

    def tile_rows(self, tile: int) -> int:
        return _load().gpa_tile_rows(_ptr(self.g), int(tile))


def window_1d(n: int, M: int) -> float:
    """The oracle's per-dimension window value at offset n of a nominal extent M."""
    return _load().gpa_window_1d(int(n), int(M))


def threads() -> int:
    return _load().gpa_oracle_threads()


def forward(geo: Geometry, q, k, v) -> np.ndarray:
    """Out = GPA(Q, K, V), FP64."""
    q, k, v = _f64(q), _f64(k), _f64(v)
    assert q.shape == k.shape == v.shape == geo.shape, (q.shape, geo.shape)
    out = np.empty(geo.shape, dtype=np.float64)
    _load().gpa_forward(_ptr(geo.g), WINDOWS[geo.window], geo.scale, _ptr(q), _ptr(k), _ptr(v), _ptr(out))
    return out


def backward(geo: Geometry, q, k, v, dout):
    """(dQ, dK, dV) of the loss sum(Out * dout), FP64."""
    q, k, v, dout = _f64(q), _f64(k), _f64(v), _f64(dout)
    assert q.shape == k.shape == v.shape == dout.shape == geo.shape
    dq = np.empty(geo.shape, dtype=np.float64)
    dk = np.empty_like(dq)
    dv = np.empty_like(dq)
    _load().gpa_backward(
        _ptr(geo.g), WINDOWS[geo.window], geo.scale, _ptr(q), _ptr(k), _ptr(v), _ptr(dout), _ptr(dq), _ptr(dk), _ptr(dv)
    )
    return dq, dk, dv


def _flat_rows(geo: Geometry, rows) -> np.ndarray:
    """rows: int array of (b, h, i) triples -> flat ((b*nh + h)*N + i) int64."""
    rows = np.asarray(rows, dtype=np.int64).reshape(-1, 3)
    return np.ascontiguousarray((rows[:, 0] * geo.nh + rows[:, 1]) * geo.N + rows[:, 2])


def forward_rows(geo: Geometry, q, k, v, rows, dout=None):
    """Out (and dQ if dout is given) at sampled (b, h, i) rows; [n, d] each."""
    q, k, v = _f64(q), _f64(k), _f64(v)
    flat = _flat_rows(geo, rows)
    n = flat.shape[0]
    out = np.empty((n, geo.d), dtype=np.float64)
    dq = np.empty((n, geo.d), dtype=np.float64) if dout is not None else None
    dout_p = None
    if dout is not None:
        dout = _f64(dout)
        dout_p = _ptr(dout)
    _load().gpa_rows(
        _ptr(geo.g), WINDOWS[geo.window], geo.scale, _ptr(q), _ptr(k), _ptr(v), dout_p, n, _ptr(flat), _ptr(out),
        _ptr(dq) if dq is not None else None,
    )
    return (out, dq) if dout is not None else out


def key_rows(geo: Geometry, q, k, v, dout, keys):
    """(dK, dV) at sampled (b, h, j) key rows; [n, d] each."""
    q, k, v, dout = _f64(q), _f64(k), _f64(v), _f64(dout)
    flat = _flat_rows(geo, keys)
    n = flat.shape[0]
    dk = np.empty((n, geo.d), dtype=np.float64)
    dv = np.empty((n, geo.d), dtype=np.float64)
    _load().gpa_key_rows(
        _ptr(geo.g), WINDOWS[geo.window], geo.scale, _ptr(q), _ptr(k), _ptr(v), _ptr(dout), n, _ptr(flat), _ptr(dk), _ptr(dv)
    )
    return dk, dv


def unit_fwd_bwd(geo: Geometry, q, k, v, dout, bh: int, tile: int, r0: int, r1: int) -> None:
    """Per-tile forward and backward of query rows [r0, r1) of one
    (batch*head, tile) unit; used to time the oracle on a bounded sample."""
    _load().gpa_unit_fwd_bwd(
        _ptr(geo.g), WINDOWS[geo.window], geo.scale, _ptr(q), _ptr(k), _ptr(v), _ptr(dout), int(bh), int(tile), int(r0), int(r1)
    )
