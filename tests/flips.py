"""Test helper: Gaussians that two projections composite differently (see
flips.c).  Built with gcc next to this file on first use."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "flips.c")
OUT = os.path.join(HERE, "_flips.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(OUT) or os.path.getmtime(OUT) < os.path.getmtime(SRC):
            subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", SRC, "-o", OUT, "-lm"], check=True)
        L = C.CDLL(OUT)
        D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
        L.flips.argtypes = [C.c_int, C.c_int64, I32, I32, C.c_int, D, U32, U32, D, U32, U32, U8]
        L.flips.restype = C.c_int64
        L.decision_margins.argtypes = [C.c_int, C.c_int64, I32, I32, C.c_int, D, U32, U32, D]
        L.same_sequences.argtypes = [C.c_int, C.c_int64, I32, I32, C.c_int, D, U32, U32, D, U32, U32, U8]
        L.same_sequences.restype = C.c_int64
        _lib = L
    return _lib


def decision_flips(cams, projA, valsA, rangesA, projB, valsB, rangesB, tile: int = 16):
    """Gaussians (per view) kept at some pixel under one projection and not the
    other; returns (flags [V][n] bool, number of pixels that differ)."""
    projA = np.ascontiguousarray(projA, dtype=np.float64)
    projB = np.ascontiguousarray(projB, dtype=np.float64)
    V, n = projA.shape[:2]
    flags = np.zeros(V * n, dtype=np.uint8)
    w = np.ascontiguousarray(cams["width"], dtype=np.int32)
    h = np.ascontiguousarray(cams["height"], dtype=np.int32)
    npix = _load().flips(V, n, w, h, tile, projA, np.ascontiguousarray(valsA, dtype=np.uint32),
                         np.ascontiguousarray(rangesA, dtype=np.uint32), projB,
                         np.ascontiguousarray(valsB, dtype=np.uint32),
                         np.ascontiguousarray(rangesB, dtype=np.uint32), flags)
    return flags.reshape(V, n).astype(bool), int(npix)


def decision_margins(cams, proj, vals, ranges, tile: int = 16):
    """Per pixel (views concatenated): the smallest relative distance of a
    compositing decision of its double-precision walk from its threshold
    (see flips.c); 1e300 where the list is empty."""
    proj = np.ascontiguousarray(proj, dtype=np.float64)
    V, n = proj.shape[:2]
    w = np.ascontiguousarray(cams["width"], dtype=np.int32)
    h = np.ascontiguousarray(cams["height"], dtype=np.int32)
    out = np.zeros(int(np.sum(w.astype(np.int64) * h)), dtype=np.float64)
    _load().decision_margins(V, n, w, h, tile, proj, np.ascontiguousarray(vals, dtype=np.uint32),
                             np.ascontiguousarray(ranges, dtype=np.uint32), out)
    return out


def same_sequences(cams, projA, valsA, rangesA, projB, valsB, rangesB, tile: int = 16):
    """Per pixel (views concatenated): True where the two projections' walks
    keep the same fragments in the same order (see flips.c)."""
    projA = np.ascontiguousarray(projA, dtype=np.float64)
    projB = np.ascontiguousarray(projB, dtype=np.float64)
    V, n = projA.shape[:2]
    w = np.ascontiguousarray(cams["width"], dtype=np.int32)
    h = np.ascontiguousarray(cams["height"], dtype=np.int32)
    out = np.zeros(int(np.sum(w.astype(np.int64) * h)), dtype=np.uint8)
    _load().same_sequences(V, n, w, h, tile, projA, np.ascontiguousarray(valsA, dtype=np.uint32),
                           np.ascontiguousarray(rangesA, dtype=np.uint32), projB,
                           np.ascontiguousarray(valsB, dtype=np.uint32),
                           np.ascontiguousarray(rangesB, dtype=np.uint32), out)
    return out.astype(bool)
