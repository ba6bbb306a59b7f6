"""Exact O(N^2) lattice sum (Eq. dpoissonsoln) through the C helper direct.c.

TEST INFRASTRUCTURE ONLY (see the package header).

``build()`` compiles direct.c with gcc (-O2 -fopenmp, no fast-math so the
compensated summation survives) into oracle/_build/.  Pinned by
tests/test_oracle_direct.py: a pure-Python double loop on a tiny case, and the
identity L u = f on the interior of the active grid.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

from . import lgf as _lgf

_HERE = pathlib.Path(__file__).resolve().parent
_SRC = _HERE / "direct.c"
_LIB = _HERE / "_build" / "liblgf_direct.so"
_handle = None


def build(force: bool = False) -> pathlib.Path:
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        _LIB.parent.mkdir(parents=True, exist_ok=True)
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               str(_SRC), "-o", str(tmp)])
        os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    if _handle is None:
        build()
        h = ctypes.CDLL(str(_LIB))
        h.lgf_direct_sum.restype = ctypes.c_int
        h.lgf_direct_sum.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _handle = h
    return _handle


def point_coords(blocks: np.ndarray, n_b: int) -> np.ndarray:
    """(n_blocks*n_b^3, 3) grid coordinates in block order, x fastest in a block."""
    r = np.arange(n_b)
    kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
    b = np.asarray(blocks, dtype=np.int64)[:, None, None, None, :] * n_b
    c = np.stack([ii, jj, kk], axis=-1)[None] + b
    return c.reshape(-1, 3).astype(np.int32)


def direct_sum(blocks, n_b: int, f, targets=None) -> np.ndarray:
    """u at the target points (default: all active points, shaped like f)."""
    pts = point_coords(blocks, n_b)
    fv = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
    tg = pts if targets is None else np.ascontiguousarray(np.asarray(targets, dtype=np.int32))
    span = np.maximum(pts.max(0), tg.max(0)) - np.minimum(pts.min(0), tg.min(0))
    V = int(span.max())
    tab = np.ascontiguousarray(_lgf.lgf_abs_table(1, V))
    u = np.empty(len(tg))
    rc = _lib().lgf_direct_sum(pts.ctypes.data, fv.ctypes.data, len(pts), tab.ctypes.data, V,
                               tg.ctypes.data, len(tg), u.ctypes.data)
    if rc != 0:
        raise RuntimeError("direct sum: offset outside the G table")
    return u.reshape(np.shape(f)) if targets is None else u


def stencil_residual(blocks, n_b: int, u, f) -> float:
    """max |L u - f| over the interior of the active grid (points whose six
    neighbours are all active), relative to max |f|: the discrete Poisson
    equation L u = f (Eq. dpoisson, 7-point Laplacian, unit spacing) that
    u = G * f solves exactly at every lattice point."""
    blocks = np.asarray(blocks, dtype=np.int64)
    lo = blocks.min(axis=0) * n_b - 1
    hi = (blocks.max(axis=0) + 1) * n_b + 1
    shape = tuple(int(v) for v in (hi - lo)[::-1])       # (z, y, x) with a one-point margin
    pts = point_coords(blocks, n_b).astype(np.int64) - lo
    xs, ys, zs = pts[:, 0], pts[:, 1], pts[:, 2]
    U = np.zeros(shape)
    F = np.zeros(shape)
    active = np.zeros(shape, dtype=bool)
    U[zs, ys, xs] = np.asarray(u, dtype=np.float64).reshape(-1)
    F[zs, ys, xs] = np.asarray(f, dtype=np.float64).reshape(-1)
    active[zs, ys, xs] = True
    c = (slice(1, -1),) * 3
    interior = active[c].copy()
    lap = -6.0 * U[c]
    for ax in range(3):
        for d in (0, 2):
            sl = [slice(1, -1)] * 3
            sl[ax] = slice(d, shape[ax] - 2 + d)
            lap = lap + U[tuple(sl)]
            interior &= active[tuple(sl)]
    r = np.abs(lap - F[c])[interior]
    return float(r.max() / np.abs(F).max()) if r.size else 0.0
