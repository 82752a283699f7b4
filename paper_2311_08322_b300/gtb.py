"""Thin ctypes binding of libgtb (include/gtb.h) plus the storage allocator.

Argument marshalling only: every step of hdiff / vadv runs in the CUDA
kernels of ``libgtb.so``.  PyTorch provides device memory and streams.  There
is no fallback: if the library is missing or a call fails, this module raises.

Storages (the GT4Py paper's ``storage``, Sec. 2.2/2.3) are torch tensors shaped
``(nk, nj, ni)`` (i contiguous) whose rows are padded so every interior row
starts on a 128-byte boundary and every pitch is a multiple of 128 bytes (the
TMA and vector-access layout); ``origin`` is the storage index ``(i, j, k)``
of the compute domain's first point.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# GTB_CHECKED=1 in the environment loads the checked build (libgtb_checked.so): the same
# kernels, each testing its address runs against the fields' storages first; a run
# outside them is not accessed and device_status() raises GTB_ERR_DEVICE
LIB_PATH = os.path.join(_PKG, "libgtb_checked.so" if os.environ.get("GTB_CHECKED") == "1" else "libgtb.so")

GTB_F32, GTB_F64 = 1, 2
PREC = {"native": 0, "f64": 1, "df": 2}
GTB_WCON_LITERAL = 1
STATUS = {0: "GTB_OK", -1: "GTB_ERR_NULL", -2: "GTB_ERR_DTYPE", -3: "GTB_ERR_EXTENT", -4: "GTB_ERR_LAYOUT",
          -5: "GTB_ERR_ALIAS", -6: "GTB_ERR_LAUNCH", -7: "GTB_ERR_DEVICE", -8: "GTB_ERR_UNSUPPORTED",
          -9: "GTB_ERR_ARG"}


class GtbField(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 3), ("strides", ctypes.c_int64 * 3), ("origin", ctypes.c_int64 * 3)]


class GtbMember(ctypes.Structure):
    _fields_ = [("in_", GtbField), ("coeff", GtbField), ("h", GtbField), ("wcon", GtbField), ("utens", GtbField),
                ("utens_stage", GtbField), ("out", GtbField), ("domain", ctypes.c_int64 * 3)]


class GtbBatchConfig(ctypes.Structure):
    _fields_ = [("hdiff_tile", ctypes.c_int32), ("hdiff_levels", ctypes.c_int32), ("vadv_warps", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]


class GtbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None
EXPORTS = ("gtb_hdiff", "gtb_vadv", "gtb_vadv_workspace_bytes", "gtb_hdiff_adj", "gtb_vadv_adj",
           "gtb_vadv_adj_workspace_bytes", "gtb_halo_periodic", "gtb_halo_periodic_adj", "gtb_device_status",
           "gtb_batch_plan", "gtb_batch_run", "gtb_plan_info", "gtb_plan_destroy", "gtb_hdiff_vadv",
           "gtb_hdiff_vadv_workspace_bytes", "gtb_step", "gtb_selftest_wait", "gtb_probe_fp64_fma",
           "gtb_vadv_noalloc", "gtb_last_error", "gtb_version")
GTB_ADJ_ACCUMULATE = 2
GTB_SAVE_FACTORS = 4
GTB_ADJ_FACTORS = 8
GTB_STATE48 = 16


def lib() -> ctypes.CDLL:
    """Load libgtb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2311_08322_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(GtbField)
        i64p, vp = ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p
        L.gtb_hdiff.argtypes = [P, P, P, i64p, vp]
        L.gtb_vadv.argtypes = [P, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint,
                               i64p, vp, ctypes.c_size_t, vp]
        L.gtb_vadv_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, i64p]
        L.gtb_vadv_workspace_bytes.restype = ctypes.c_size_t
        L.gtb_hdiff_adj.argtypes = [P, P, P, P, P, ctypes.c_uint, i64p, vp]
        L.gtb_vadv_adj.argtypes = [P, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint,
                                   i64p, vp, ctypes.c_size_t, vp]
        L.gtb_vadv_adj_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, i64p]
        L.gtb_vadv_adj_workspace_bytes.restype = ctypes.c_size_t
        L.gtb_hdiff_vadv.argtypes = [P, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_uint, i64p, vp, ctypes.c_size_t, vp]
        L.gtb_hdiff_vadv.restype = ctypes.c_int
        L.gtb_step.argtypes = [P, P, P, P, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_uint, i64p, vp, ctypes.c_size_t, vp]
        L.gtb_step.restype = ctypes.c_int
        L.gtb_hdiff_vadv_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint, i64p]
        L.gtb_hdiff_vadv_workspace_bytes.restype = ctypes.c_size_t
        L.gtb_halo_periodic.argtypes = [P, ctypes.c_int, ctypes.c_int, i64p, vp]
        L.gtb_halo_periodic_adj.argtypes = [P, ctypes.c_int, ctypes.c_int, i64p, vp]
        for n in ("gtb_hdiff_adj", "gtb_vadv_adj", "gtb_halo_periodic", "gtb_halo_periodic_adj"):
            getattr(L, n).restype = ctypes.c_int
        L.gtb_batch_plan.argtypes = [ctypes.POINTER(GtbMember), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_uint, ctypes.POINTER(GtbBatchConfig),
                                     ctypes.POINTER(ctypes.c_void_p)]
        L.gtb_batch_run.argtypes = [ctypes.c_void_p, vp]
        L.gtb_plan_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        L.gtb_plan_destroy.argtypes = [ctypes.c_void_p]
        for n in ("gtb_batch_plan", "gtb_batch_run", "gtb_plan_info", "gtb_plan_destroy"):
            getattr(L, n).restype = ctypes.c_int
        L.gtb_device_status.argtypes = [vp]
        L.gtb_selftest_wait.argtypes = [ctypes.c_longlong, ctypes.c_int, vp]
        L.gtb_selftest_wait.restype = ctypes.c_int
        L.gtb_probe_fp64_fma.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp]
        L.gtb_probe_fp64_fma.restype = ctypes.c_int
        L.gtb_vadv_noalloc.argtypes = [P, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_uint, i64p, vp]
        L.gtb_vadv_noalloc.restype = ctypes.c_int
        L.gtb_last_error.restype = ctypes.c_char_p
        L.gtb_version.restype = ctypes.c_char_p
        for n in ("gtb_hdiff", "gtb_vadv", "gtb_device_status"):
            getattr(L, n).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise GtbError(rc, lib().gtb_last_error().decode())


def version() -> str:
    return lib().gtb_version().decode()


# ----------------------------------------------------------------- storages
@dataclass
class Storage:
    """A field storage: ``data`` (torch, shaped (nk, nj, ni)) and its ``origin``."""
    data: torch.Tensor
    origin: tuple

    @property
    def shape(self):
        return tuple(self.data.shape)

    def numpy(self) -> np.ndarray:
        return self.data.detach().cpu().numpy().copy()

    def interior(self, domain) -> torch.Tensor:
        (oi, oj, ok), (I, J, K) = self.origin, domain
        return self.data[ok:ok + K, oj:oj + J, oi:oi + I]


def empty_storage(ni: int, nj: int, nk: int, *, dtype=torch.float64, device="cuda", halo_i: int = 0,
                  align_bytes: int = 128) -> torch.Tensor:
    """Padded (nk, nj, ni) tensor: storage column ``halo_i`` of every row is
    ``align_bytes``-aligned and the row pitch is a multiple of ``align_bytes``."""
    es = torch.empty((), dtype=dtype).element_size()
    a = align_bytes // es
    lead = (-halo_i) % a
    sj = -(-(lead + ni) // a) * a
    sk = sj * nj
    n = max(1, nk * sk)
    buf = torch.empty(n + 2 * a, dtype=dtype, device=device)
    # the caching allocator returns 512-byte-aligned blocks; keep `lead` from there
    off = ((-buf.data_ptr() // es) % a) + lead
    return buf.as_strided((nk, nj, ni), (sk, sj, 1), storage_offset=off)


def storage_from(arr: np.ndarray, origin, *, device="cuda", dtype=None) -> Storage:
    """Copy a host (nk, nj, ni) array into a padded device storage."""
    dt = dtype or (torch.float32 if arr.dtype == np.float32 else torch.float64)
    nk, nj, ni = arr.shape
    t = empty_storage(ni, nj, nk, dtype=dt, device=device, halo_i=origin[0])
    t.copy_(torch.from_numpy(np.ascontiguousarray(arr)).to(dt))
    return Storage(t, tuple(origin))


def field(t, origin=None) -> GtbField:
    """gtb_field describing a CUDA tensor (or Storage) shaped (nk, nj, ni).  A Storage
    keeps the descriptor it was last given and reuses it while its tensor's pointer,
    dtype, shape and strides and its origin are unchanged (building the ctypes
    structure is most of a call's Python cost)."""
    if isinstance(t, Storage):
        if origin is None:
            d = t.data
            key = (d.data_ptr(), d.dtype, d.shape, d.stride(), t.origin)
            memo = t.__dict__.get("_field_memo")
            if memo is not None and memo[0] == key:
                return memo[1]
            f = field(d, t.origin)
            t.__dict__["_field_memo"] = (key, f)
            return f
        t = t.data
    if origin is None:
        origin = (0, 0, 0)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("gtb fields must be CUDA tensors")
    if t.dim() != 3:
        raise ValueError("gtb fields are 3-D tensors shaped (nk, nj, ni)")
    if t.dtype == torch.float64:
        dt = GTB_F64
    elif t.dtype == torch.float32:
        dt = GTB_F32
    else:
        raise TypeError(f"unsupported dtype {t.dtype}")
    nk, nj, ni = t.shape
    sk, sj, si = t.stride()
    f = GtbField()
    f.ptr = t.data_ptr()
    f.dtype = dt
    f.reserved = 0
    f.shape[:] = [ni, nj, nk]
    f.strides[:] = [si, sj, sk]
    f.origin[:] = list(origin)
    return f


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dom(domain):
    if domain is None:
        return None
    return (ctypes.c_int64 * 3)(*[int(x) for x in domain])


# ----------------------------------------------------------------- stencils
def hdiff(in_, coeff, out, *, domain=None, stream=None):
    """out = hdiff(in_, coeff) on the domain (gtb_hdiff).  Fields: Storage or
    (tensor, origin) pairs.  Asynchronous on ``stream`` (default: torch's current)."""
    fi, fc, fo = (_as_field(x) for x in (in_, coeff, out))
    _check(lib().gtb_hdiff(ctypes.byref(fi), ctypes.byref(fc), ctypes.byref(fo), _dom(domain), _stream(stream)))
    return out


def vadv_workspace_bytes(dtype, prec, domain) -> int:
    """Workspace bytes gtb_vadv uses for this storage dtype, prec and domain (I, J, K)."""
    dt = {torch.float64: GTB_F64, torch.float32: GTB_F32}.get(dtype, dtype)
    return int(lib().gtb_vadv_workspace_bytes(dt, PREC[prec] if isinstance(prec, str) else int(prec), _dom(domain)))


_ws_cache = {}


def workspace(nbytes: int, stream=None) -> torch.Tensor:
    """A cached device scratch buffer of at least ``nbytes`` bytes for one (device, stream):
    calls that may run concurrently on different streams get different buffers."""
    key = (torch.cuda.current_device(), _stream(stream).value)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
        _ws_cache[key] = buf
    return buf


def _vadv_domain(fs, literal):
    """Deduced domain: the largest keeping every access inside its storage (paper Sec. 2.2)."""
    dom = []
    for d in range(3):
        reach = [1 if (q == 1 and d == 0 and not literal) else 0 for q in range(6)]
        dom.append(min(f.shape[d] - f.origin[d] - r for f, r in zip(fs, reach)))
    return tuple(max(0, x) for x in dom)


def vadv(u_stage, wcon, u_pos, utens, utens_stage, out=None, *, dtr_stage=3.0 / 20.0, beta_v=0.0,
         prec="native", literal=False, domain=None, workspace="auto", state48=False, stream=None):
    """utens_stage_out = vadv(...) (gtb_vadv); ``out=None`` updates utens_stage in place.

    ``workspace``: "auto" (a cached buffer from :func:`workspace`, the fast
    form), a CUDA tensor, or None (column state in shared memory).
    ``state48``: GTB_STATE48 (FP32 storage, prec "df": the column state in 48 bits)."""
    out = utens_stage if out is None else out
    fs = [_as_field(x) for x in (u_stage, wcon, u_pos, utens, utens_stage, out)]
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        if isinstance(workspace, str):
            dom = tuple(domain) if domain is not None else _vadv_domain(fs, literal)
            need = vadv_workspace_bytes(fs[0].dtype, prec, dom)
            workspace = globals()["workspace"](need, stream) if need else None
        if workspace is not None:
            ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib().gtb_vadv(*[ctypes.byref(f) for f in fs], float(dtr_stage), float(beta_v),
                          PREC[prec] if isinstance(prec, str) else int(prec),
                          (GTB_WCON_LITERAL if literal else 0) | (GTB_STATE48 if state48 else 0),
                          _dom(domain), ctypes.c_void_p(ws_ptr) if ws_ptr else None, ws_bytes, _stream(stream)))
    return out


def _fused_domain(fs, literal):
    """Deduced domain of hdiff_vadv: in needs 2 halo points in I and J, wcon one above I."""
    dom = []
    for d in range(3):
        reach = [2 if d < 2 else 0] + [0] * 5
        if d == 0 and not literal:
            reach[2] = 1
        dom.append(min(f.shape[d] - f.origin[d] - r for f, r in zip(fs, reach)))
    return tuple(max(0, x) for x in dom)


def hdiff_vadv_workspace_bytes(dtype, prec, domain, save_factors=False) -> int:
    """Workspace bytes gtb_hdiff_vadv needs (with room for the kept factors when asked)."""
    dt = {torch.float64: GTB_F64, torch.float32: GTB_F32}.get(dtype, dtype)
    return int(lib().gtb_hdiff_vadv_workspace_bytes(dt, PREC[prec] if isinstance(prec, str) else int(prec),
                                                    GTB_SAVE_FACTORS if save_factors else 0, _dom(domain)))


def hdiff_vadv(in_, coeff, wcon, utens, utens_stage, out=None, *, dtr_stage=3.0 / 20.0, beta_v=0.0,
               prec="native", literal=False, domain=None, workspace="auto", save_factors=False, stream=None):
    """utens_stage_out = vadv(h, wcon, h, utens, utens_stage) with h = hdiff(in_, coeff), in one
    kernel (gtb_hdiff_vadv); ``out=None`` updates utens_stage in place.  ``workspace``: "auto"
    (a cached buffer from :func:`workspace`) or a CUDA tensor; the call needs one.  With
    ``save_factors`` the workspace keeps the column factors for :func:`vadv_adj` (``factors=True``):
    pass a tensor of :func:`hdiff_vadv_workspace_bytes` bytes that outlives the call."""
    out = utens_stage if out is None else out
    fs = [_as_field(x) for x in (in_, coeff, wcon, utens, utens_stage, out)]
    ws_ptr, ws_bytes = None, 0
    if isinstance(workspace, str):
        dom = tuple(domain) if domain is not None else _fused_domain(fs, literal)
        need = hdiff_vadv_workspace_bytes(fs[0].dtype, prec, dom, save_factors)
        workspace = globals()["workspace"](need, stream) if need else None
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    flags = (GTB_WCON_LITERAL if literal else 0) | (GTB_SAVE_FACTORS if save_factors else 0)
    _check(lib().gtb_hdiff_vadv(*[ctypes.byref(f) for f in fs], float(dtr_stage), float(beta_v),
                                PREC[prec] if isinstance(prec, str) else int(prec), flags, _dom(domain),
                                ctypes.c_void_p(ws_ptr) if ws_ptr else None, ws_bytes, _stream(stream)))
    return out


def step(in_, coeff, hdiff_out, u_stage, wcon, u_pos, utens, utens_stage, out=None, *, dtr_stage=3.0 / 20.0,
         beta_v=0.0, prec="native", literal=False, domain=None, workspace="auto", state48=False, stream=None):
    """Both benchmark stencils on their own fields in one co-scheduled kernel (gtb_step):
    hdiff_out = hdiff(in_, coeff); out = vadv(u_stage, wcon, u_pos, utens, utens_stage)
    (``out=None`` updates utens_stage in place).  ``workspace``: "auto" or a CUDA tensor.
    ``state48``: as :func:`vadv`."""
    out = utens_stage if out is None else out
    fs = [_as_field(x) for x in (in_, coeff, hdiff_out, u_stage, wcon, u_pos, utens, utens_stage, out)]
    ws_ptr, ws_bytes = None, 0
    if isinstance(workspace, str):
        # deduced domain: in reaches 2 points in I and J, wcon one point above I
        reach = [(2, 2, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), (0 if literal else 1, 0, 0)] + [(0, 0, 0)] * 4
        dom = tuple(domain) if domain is not None else tuple(
            max(0, min(f.shape[d] - f.origin[d] - r[d] for f, r in zip(fs, reach))) for d in range(3))
        need = vadv_workspace_bytes(fs[0].dtype, prec, dom)
        workspace = globals()["workspace"](need, stream) if need else None
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib().gtb_step(*[ctypes.byref(f) for f in fs], float(dtr_stage), float(beta_v),
                          PREC[prec] if isinstance(prec, str) else int(prec),
                          (GTB_WCON_LITERAL if literal else 0) | (GTB_STATE48 if state48 else 0),
                          _dom(domain), ctypes.c_void_p(ws_ptr) if ws_ptr else None, ws_bytes, _stream(stream)))
    return out


def _ptr(x):
    return None if x is None else ctypes.byref(_as_field(x))


def hdiff_adj(in_, coeff, out_bar, in_bar, coeff_bar=None, *, accumulate=False, domain=None, stream=None):
    """Reverse-mode hdiff (gtb_hdiff_adj): in_bar on the domain plus its 2-ring,
    coeff_bar (optional) on the domain."""
    _check(lib().gtb_hdiff_adj(_ptr(in_), _ptr(coeff), _ptr(out_bar), _ptr(in_bar), _ptr(coeff_bar),
                               GTB_ADJ_ACCUMULATE if accumulate else 0, _dom(domain), _stream(stream)))
    return in_bar


def vadv_adj(wcon, y_bar, u_stage_bar=None, u_pos_bar=None, utens_bar=None, utens_stage_bar=None, *,
             dtr_stage=3.0 / 20.0, beta_v=0.0, prec="native", literal=False, accumulate=False, domain=None,
             workspace="auto", factors=False, stream=None):
    """Reverse-mode vadv for fixed wcon (gtb_vadv_adj).  Passing one storage as both
    u_stage_bar and u_pos_bar stores their sum there.  ``factors=True``: ``workspace`` is the
    buffer that :func:`hdiff_vadv` filled with ``save_factors=True`` (consumed here)."""
    fw, fy = _as_field(wcon), _as_field(y_bar)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        if isinstance(workspace, str):
            dom = tuple(domain) if domain is not None else tuple(fy.shape[d] - fy.origin[d] for d in range(3))
            need = int(lib().gtb_vadv_adj_workspace_bytes(fy.dtype, PREC[prec], _dom(dom)))
            workspace = globals()["workspace"](need, stream) if need else None
        if workspace is not None:
            ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    flags = (1 if literal else 0) | (GTB_ADJ_ACCUMULATE if accumulate else 0) | (GTB_ADJ_FACTORS if factors else 0)
    _check(lib().gtb_vadv_adj(ctypes.byref(fw), ctypes.byref(fy), _ptr(u_stage_bar), _ptr(u_pos_bar),
                              _ptr(utens_bar), _ptr(utens_stage_bar), float(dtr_stage), float(beta_v), PREC[prec],
                              flags, _dom(domain), ctypes.c_void_p(ws_ptr) if ws_ptr else None, ws_bytes,
                              _stream(stream)))


def halo_periodic(f, hi=2, hj=2, *, domain=None, stream=None):
    """Periodic refresh of the hi x hj halo around the domain (gtb_halo_periodic)."""
    _check(lib().gtb_halo_periodic(_ptr(f), int(hi), int(hj), _dom(domain), _stream(stream)))
    return f


def halo_periodic_adj(f, hi=2, hj=2, *, domain=None, stream=None):
    """Adjoint of the refresh: fold the halo's values into the domain (gtb_halo_periodic_adj)."""
    _check(lib().gtb_halo_periodic_adj(_ptr(f), int(hi), int(hj), _dom(domain), _stream(stream)))
    return f


def selftest_wait(limit_ns: int, arrive: bool, stream=None):
    """Exercise the bounded-wait failure path (gtb_selftest_wait): with arrive=False the
    wait runs out after limit_ns and device_status() then raises GTB_ERR_DEVICE."""
    _check(lib().gtb_selftest_wait(int(limit_ns), 1 if arrive else 0, _stream(stream)))


def probe_fp64_fma(blocks: int, iters: int, sink: torch.Tensor, stream=None):
    """Launch the FP64 FMA issue-rate probe (gtb_probe_fp64_fma): blocks * 256 * 8 * iters
    binary64 FMAs; the caller times it."""
    _check(lib().gtb_probe_fp64_fma(int(blocks), int(iters), ctypes.c_void_p(sink.data_ptr()), _stream(stream)))
    return blocks * 256 * 8 * iters


def device_status(stream=None):
    """Synchronise the stream and raise if a kernel's bounded wait expired."""
    _check(lib().gtb_device_status(_stream(stream)))


def _as_field(x) -> GtbField:
    if isinstance(x, GtbField):
        return x
    if isinstance(x, Storage):
        return field(x)
    if isinstance(x, tuple) and len(x) == 2:
        return field(x[0], x[1])
    raise TypeError("expected a Storage, a (tensor, origin) pair or a GtbField")


# ----------------------------------------------------------------- batched ensembles
DEFAULT_BATCH_CONFIG = {"hdiff_tile": 0, "hdiff_levels": 8, "vadv_warps": 2, "ctas_per_sm": 0}
MEMBER_FIELDS = ("in", "coeff", "h", "wcon", "utens", "utens_stage", "out")


class BatchPlan:
    """A validated ensemble captured into a CUDA graph (gtb_batch_plan).

    ``members``: dicts with Storages under MEMBER_FIELDS and ``domain`` (I, J, K).
    Each member runs h = hdiff(in, coeff) then out = vadv(h, wcon, h, utens,
    utens_stage).  ``run()`` replays the graph on a stream; the plan keeps its
    members' storages alive."""

    def __init__(self, members, *, dtr_stage=3.0 / 20.0, beta_v=0.0, prec="native", literal=False, config=None):
        self.members = members
        arr = (GtbMember * len(members))()
        for q, m in enumerate(members):
            for name in MEMBER_FIELDS:
                setattr(arr[q], "in_" if name == "in" else name, field(m[name]))
            arr[q].domain[:] = [int(x) for x in m["domain"]]
        self.config = dict(DEFAULT_BATCH_CONFIG, **(config or {}))
        cfg = GtbBatchConfig(**self.config)
        h = ctypes.c_void_p()
        _check(lib().gtb_batch_plan(arr, len(members), float(dtr_stage), float(beta_v), PREC[prec],
                                    1 if literal else 0, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(lib().gtb_batch_run(self._h, _stream(stream)))

    def info(self) -> dict:
        v = (ctypes.c_int64 * 6)()
        _check(lib().gtb_plan_info(self._h, v))
        return dict(zip(("hdiff_items", "vadv_items", "hdiff_grid", "vadv_grid", "points", "members"), list(v)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gtb_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def member_storages(fields: dict, I: int, J: int, K: int, device="cuda") -> dict:
    """Device storages of one ensemble member from its seeded draws (hdiff halo 2,
    vadv halo 1, h interior, out with halo 1)."""
    o2, o1 = (2, 2, 0), (1, 1, 0)
    m = {"in": storage_from(fields["in"], o2, device=device), "coeff": storage_from(fields["coeff"], o2, device=device)}
    for n in ("wcon", "utens", "utens_stage"):
        m[n] = storage_from(fields[n], o1, device=device)
    dt = torch.float32 if fields["in"].dtype == np.float32 else torch.float64
    m["h"] = Storage(empty_storage(I, J, K, dtype=dt, device=device), (0, 0, 0))
    m["out"] = Storage(empty_storage(I + 2, J + 2, K, dtype=dt, device=device, halo_i=1), o1)
    m["domain"] = (I, J, K)
    return m


def run_member_single(m, *, dtr_stage=3.0 / 20.0, beta_v=0.0, prec="native", stream=None):
    """The same member with the single-domain entry points (gtb_hdiff, gtb_vadv)."""
    hdiff(m["in"], m["coeff"], m["h"], domain=m["domain"], stream=stream)
    vadv(m["h"], m["wcon"], m["h"], m["utens"], m["utens_stage"], m["out"], dtr_stage=dtr_stage, beta_v=beta_v,
         prec=prec, domain=m["domain"], stream=stream)
