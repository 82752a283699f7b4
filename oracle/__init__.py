"""CPU oracle for the hdiff / vadv stencils (GT4Py paper, Sec. 3.1).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  The arithmetic
lives in ``gtb_oracle.c`` (plain loops, binary64, ``-ffp-contract=off``); this
module only compiles it with gcc, loads it with ctypes and marshals numpy
arrays.  It imports nothing from the CUDA package.

Arrays are numpy float64, C-contiguous, shaped ``(nk, nj, ni)`` (i fastest),
i.e. whole storages including halos.  ``origin`` is the storage index
``(i, j, k)`` of compute-domain point (0,0,0) and ``domain`` is ``(I, J, K)``
(the paper's ``origin``/``domain`` call arguments, Sec. 2.2).  Reduced-precision
inputs are widened to float64 by the caller before they reach the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gtb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gtb_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _OField(ctypes.Structure):
    _fields_ = [("p", ctypes.c_void_p), ("ni", ctypes.c_int64), ("nj", ctypes.c_int64),
                ("nk", ctypes.c_int64), ("oi", ctypes.c_int64), ("oj", ctypes.c_int64),
                ("ok", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        # GTB_ORACLE_LIB lets the mutation tests load a deliberately broken copy.
        lib = ctypes.CDLL(os.environ.get("GTB_ORACLE_LIB") or build())
        P = ctypes.POINTER(_OField)
        i64, dbl, dp = ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
        lib.oracle_hdiff.argtypes = [P, P, P, i64, i64, i64]
        lib.oracle_vadv.argtypes = [P, P, P, P, P, P, i64, i64, i64, dbl, dbl, ctypes.c_int]
        lib.oracle_vadv_system.argtypes = [P, P, P, P, P, i64, i64, i64, dbl, dbl, ctypes.c_int,
                                           dp, dp, dp, dp]
        lib.oracle_thomas.argtypes = [dp, dp, dp, dp, i64, dp, dp, dp]
        lib.oracle_thomas_ld.argtypes = [dp, dp, dp, dp, i64, dp]
        lib.oracle_hdiff_adj.argtypes = [P, P, P, P, P, i64, i64, i64]
        lib.oracle_vadv_adj.argtypes = [P, P, P, P, P, P, i64, i64, i64, dbl, dbl, ctypes.c_int]
        for f in (lib.oracle_hdiff, lib.oracle_vadv, lib.oracle_vadv_system, lib.oracle_thomas,
                  lib.oracle_thomas_ld, lib.oracle_hdiff_adj, lib.oracle_vadv_adj):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a: np.ndarray) -> np.ndarray:
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.ndim != 3:
        raise TypeError("oracle fields must be C-contiguous float64 arrays shaped (nk, nj, ni)")
    return a


def _ofield(a: np.ndarray, origin) -> _OField:
    nk, nj, ni = a.shape
    oi, oj, ok = origin
    return _OField(a.ctypes.data, ni, nj, nk, oi, oj, ok)


def _check_extent(name, a, origin, domain, lo=(0, 0, 0), hi=(0, 0, 0)):
    nk, nj, ni = a.shape
    for d, (o, n, s, l, h) in enumerate(zip(origin, domain, (ni, nj, nk), lo, hi)):
        if o - l < 0 or o + n + h > s:
            raise ValueError(f"{name}: domain plus its stencil reach leaves the storage in axis {d}")


def hdiff(inp, coeff, out=None, *, origin_in=(2, 2, 0), origin_coeff=None, origin_out=None,
          domain=None):
    """Horizontal diffusion, returns ``out`` (allocated like ``coeff`` if not given)."""
    inp, coeff = _f64(inp), _f64(coeff)
    if domain is None:
        nk, nj, ni = inp.shape
        domain = (ni - 2 * origin_in[0], nj - 2 * origin_in[1], nk - 2 * origin_in[2])
    origin_coeff = origin_in if origin_coeff is None else origin_coeff
    if out is None:
        out = np.zeros_like(coeff)
        if origin_out is None:
            origin_out = origin_coeff
    elif origin_out is None:
        origin_out = origin_in
    out = _f64(out)
    _check_extent("in", inp, origin_in, domain, (2, 2, 0), (2, 2, 0))
    _check_extent("coeff", coeff, origin_coeff, domain)
    _check_extent("out", out, origin_out, domain)
    I, J, K = domain
    fi, fc, fo = _ofield(inp, origin_in), _ofield(coeff, origin_coeff), _ofield(out, origin_out)
    if _load().oracle_hdiff(ctypes.byref(fi), ctypes.byref(fc), ctypes.byref(fo), I, J, K) != 0:
        raise MemoryError("oracle_hdiff")
    return out


def vadv(u_stage, wcon, u_pos, utens, utens_stage, out=None, *, origin=(1, 1, 0),
         origin_wcon=None, origin_out=None, domain=None, dtr_stage=3.0 / 20.0, beta_v=0.0,
         wmode=0):
    """Vertical advection (implicit, Thomas per column); returns the new ``utens_stage``.

    All fields except ``wcon`` share ``origin``; ``wcon`` additionally needs the
    point ``i+1`` (staggered in I) when ``wmode == 0``.
    """
    fields = [_f64(x) for x in (u_stage, wcon, u_pos, utens, utens_stage)]
    if domain is None:
        nk, nj, ni = fields[0].shape
        domain = (ni - 2 * origin[0], nj - 2 * origin[1], nk - 2 * origin[2])
    origin_wcon = origin if origin_wcon is None else origin_wcon
    origin_out = origin if origin_out is None else origin_out
    if out is None:
        out = np.zeros_like(fields[4])
    out = _f64(out)
    for name, a in zip(("u_stage", "u_pos", "utens", "utens_stage"),
                       (fields[0], fields[2], fields[3], fields[4])):
        _check_extent(name, a, origin, domain)
    _check_extent("wcon", fields[1], origin_wcon, domain, (0, 0, 0), (1 if wmode == 0 else 0, 0, 0))
    _check_extent("out", out, origin_out, domain)
    I, J, K = domain
    of = [_ofield(a, origin) for a in fields]
    of[1] = _ofield(fields[1], origin_wcon)
    fo = _ofield(out, origin_out)
    rc = _load().oracle_vadv(*[ctypes.byref(f) for f in of], ctypes.byref(fo), I, J, K,
                             float(dtr_stage), float(beta_v), int(wmode))
    if rc != 0:
        raise MemoryError("oracle_vadv")
    return out


def vadv_system(u_stage, wcon, u_pos, utens, utens_stage, i, j, *, origin=(1, 1, 0),
                origin_wcon=None, K=None, dtr_stage=3.0 / 20.0, beta_v=0.0, wmode=0):
    """The tridiagonal system (a, b, c, d) of column (i, j), each of length K."""
    fields = [_f64(x) for x in (u_stage, wcon, u_pos, utens, utens_stage)]
    K = fields[0].shape[0] - origin[2] if K is None else K
    origin_wcon = origin if origin_wcon is None else origin_wcon
    of = [_ofield(a, origin) for a in fields]
    of[1] = _ofield(fields[1], origin_wcon)
    a, b, c, d = (np.zeros(K) for _ in range(4))
    dp = ctypes.POINTER(ctypes.c_double)
    _load().oracle_vadv_system(*[ctypes.byref(f) for f in of], i, j, K, float(dtr_stage),
                               float(beta_v), int(wmode), *[v.ctypes.data_as(dp) for v in (a, b, c, d)])
    return a, b, c, d


def thomas(a, b, c, d, *, extended=False):
    """Solve the tridiagonal system with the oracle's Thomas recurrences.

    Returns ``x`` (binary64 path: also the pivots and c'), or with
    ``extended=True`` the x87 long-double result rounded to binary64.
    """
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    K = a.shape[0]
    x = np.zeros(K)
    dp = ctypes.POINTER(ctypes.c_double)
    ptrs = [v.ctypes.data_as(dp) for v in (a, b, c, d)]
    if extended:
        _load().oracle_thomas_ld(*ptrs, K, x.ctypes.data_as(dp))
        return x
    piv, cpr = np.zeros(K), np.zeros(K)
    _load().oracle_thomas(*ptrs, K, x.ctypes.data_as(dp), piv.ctypes.data_as(dp),
                          cpr.ctypes.data_as(dp))
    return x, piv, cpr


def hdiff_adj(inp, coeff, out_bar, *, origin=(2, 2, 0), domain=None, coeff_bar=None):
    """Reverse-mode hdiff: returns in_bar (same storage shape as ``inp``, written on
    the domain plus its 2-point ring, zero elsewhere); ``coeff_bar`` (optional,
    shaped like ``coeff``) is accumulated.  All fields share ``origin``."""
    inp, coeff, out_bar = _f64(inp), _f64(coeff), _f64(out_bar)
    if domain is None:
        nk, nj, ni = inp.shape
        domain = (ni - 2 * origin[0], nj - 2 * origin[1], nk - 2 * origin[2])
    in_bar = np.zeros_like(inp)
    _check_extent("in", inp, origin, domain, (2, 2, 0), (2, 2, 0))
    for name, a in (("coeff", coeff), ("out_bar", out_bar)):
        _check_extent(name, a, origin, domain)
    I, J, K = domain
    fs = [_ofield(a, origin) for a in (inp, coeff, out_bar, in_bar)]
    cb = None if coeff_bar is None else ctypes.byref(_ofield(_f64(coeff_bar), origin))
    if _load().oracle_hdiff_adj(*[ctypes.byref(f) for f in fs], cb, I, J, K) != 0:
        raise MemoryError("oracle_hdiff_adj")
    return in_bar


def vadv_adj(wcon, y_bar, *, origin=(1, 1, 0), origin_wcon=None, domain=None, dtr_stage=3.0 / 20.0,
             beta_v=0.0, wmode=0):
    """Reverse-mode vadv: returns (u_stage_bar, u_pos_bar, utens_bar, utens_stage_bar),
    shaped like ``y_bar``, written on the domain (wcon is held fixed)."""
    wcon, y_bar = _f64(wcon), _f64(y_bar)
    if domain is None:
        nk, nj, ni = y_bar.shape
        domain = (ni - 2 * origin[0], nj - 2 * origin[1], nk - 2 * origin[2])
    origin_wcon = origin if origin_wcon is None else origin_wcon
    _check_extent("wcon", wcon, origin_wcon, domain, (0, 0, 0), (1 if wmode == 0 else 0, 0, 0))
    _check_extent("y_bar", y_bar, origin, domain)
    outs = [np.zeros_like(y_bar) for _ in range(4)]
    I, J, K = domain
    fw = _ofield(wcon, origin_wcon)
    fo = [_ofield(a, origin) for a in (y_bar, *outs)]
    rc = _load().oracle_vadv_adj(ctypes.byref(fw), *[ctypes.byref(f) for f in fo], I, J, K, float(dtr_stage),
                                 float(beta_v), int(wmode))
    if rc != 0:
        raise MemoryError("oracle_vadv_adj")
    return tuple(outs)
