"""The C ABI (include/gtb.h): the library builds, loads and exports every
declared entry point, and the host-side argument checks (the paper's run-time
storage checks, Sec. 3.1) return their documented codes before any CUDA call.
No GPU is needed: every call here fails validation or has an empty domain."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2311_08322_b300 import build, gtb
    build.build()
    return gtb


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "gtb.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(gtb_\w+)\s*\(", hdr)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert {"gtb_hdiff", "gtb_vadv", "gtb_vadv_workspace_bytes", "gtb_device_status", "gtb_last_error",
            "gtb_version"} <= set(syms)
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_checked_build_exports_every_declared_symbol(L):
    """The checked build (GTB_CHECKED=1) is a drop-in for the default library."""
    from paper_2311_08322_b300 import build
    lib = ctypes.CDLL(build.LIB_CHECKED)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    lib.gtb_version.restype = ctypes.c_char_p
    assert lib.gtb_version().decode().endswith(" checked")


def test_version(L):
    assert L.version().startswith("gtb ")


def fake(L, ni, nj, nk, origin=(2, 2, 0), dtype=2, ptr=0x10000000, sj=None, sk=None):
    f = L.GtbField()
    f.ptr = ptr
    f.dtype = dtype
    f.shape[:] = [ni, nj, nk]
    sj = ni if sj is None else sj
    sk = sj * nj if sk is None else sk
    f.strides[:] = [1, sj, sk]
    f.origin[:] = list(origin)
    return f


def call_hdiff(L, fi, fc, fo, domain=None):
    d = None if domain is None else (ctypes.c_int64 * 3)(*domain)
    return L.lib().gtb_hdiff(ctypes.byref(fi), ctypes.byref(fc), ctypes.byref(fo), d, None)


def test_hdiff_validation(L):
    G = 1 << 24  # separate fake address ranges
    ok = lambda: (fake(L, 12, 12, 3, ptr=G), fake(L, 12, 12, 3, ptr=2 * G), fake(L, 12, 12, 3, ptr=3 * G))
    fi, fc, fo = ok()
    # empty domain: validated, nothing launched
    assert call_hdiff(L, fi, fc, fo, (0, 8, 3)) == 0
    assert L.lib().gtb_hdiff(None, ctypes.byref(fc), ctypes.byref(fo), None, None) == -1
    fi.ptr = 0
    assert call_hdiff(L, fi, fc, fo, (0, 8, 3)) == -1
    fi, fc, fo = ok()
    fc.dtype = 1
    assert call_hdiff(L, fi, fc, fo, (0, 8, 3)) == -2
    fi, fc, fo = ok()
    fi.strides[0] = 2
    assert call_hdiff(L, fi, fc, fo, (0, 8, 3)) == -4
    fi, fc, fo = ok()
    fi.origin[0] = 1          # halo of 1 < the 2-point reach of hdiff
    assert call_hdiff(L, fi, fc, fo, (0, 8, 3)) == -3
    fi, fc, fo = ok()
    assert call_hdiff(L, fi, fc, fo, (9, 8, 3)) == -3   # 2 + 9 + 2 > 12
    fi, fc, fo = ok()
    fo.ptr = fi.ptr + 8 * 100  # out inside in's storage
    assert call_hdiff(L, fi, fc, fo, (0, 8, 3)) == -5
    assert "overlaps" in L.lib().gtb_last_error().decode()


def test_hdiff_domain_deduction(L):
    """Domain deduced from the field sizes and the stencil's reach (paper Sec. 2.2):
    an in storage of 12 with origin 2 leaves room for 8 points."""
    G = 1 << 24
    fi, fc, fo = fake(L, 12, 12, 3, ptr=G), fake(L, 12, 12, 0, ptr=2 * G), fake(L, 12, 12, 3, ptr=3 * G)
    # coeff has nk = 0, so the deduced domain is empty and nothing is launched
    assert call_hdiff(L, fi, fc, fo) == 0


def test_vadv_validation(L):
    G = 1 << 24
    mk = lambda n, o=(1, 1, 0): fake(L, 10, 10, 6, origin=o, ptr=n * G)
    fs = [mk(n) for n in range(1, 7)]
    args = lambda fs, prec=0, flags=0, dom=(0, 8, 6): [*[ctypes.byref(f) for f in fs], 0.15, 0.0, prec, flags,
                                                       (ctypes.c_int64 * 3)(*dom), None, 0, None]
    assert L.lib().gtb_vadv(*args(fs)) == 0
    assert L.lib().gtb_vadv(*args(fs, prec=1)) == -9       # FP64 storage: binary64 only
    assert L.lib().gtb_vadv(*args(fs, flags=4)) == -9
    assert L.lib().gtb_vadv(*args(fs, flags=16)) == -9      # GTB_STATE48: FP32 + double-float only
    f32 = [fake(L, 10, 10, 6, origin=(1, 1, 0), dtype=1, ptr=n * G) for n in range(1, 7)]
    assert L.lib().gtb_vadv(*args(f32, prec=0, flags=16)) == -9
    assert L.lib().gtb_vadv(*args(f32, prec=1, flags=16)) == -9
    assert L.lib().gtb_vadv(*args(f32, prec=2, flags=17)) == 0  # empty domain: nothing launched
    assert L.lib().gtb_vadv(*args(fs, dom=(9, 8, 6))) == -3  # wcon needs i+1 <= 9
    assert L.lib().gtb_vadv(*args(fs, flags=1, dom=(0, 8, 6))) == 0
    big = [fake(L, 10, 10, 500, origin=(1, 1, 0), ptr=n * (1 << 28)) for n in range(1, 7)]
    assert L.lib().gtb_vadv(*args(big, dom=(8, 8, 449))) == -8
    # in place: the very same view is allowed, a shifted one is not
    fs2 = [mk(n) for n in range(1, 6)] + [mk(5)]
    assert L.lib().gtb_vadv(*args(fs2)) == 0
    fs3 = [mk(n) for n in range(1, 6)] + [mk(5, o=(1, 2, 0))]
    assert L.lib().gtb_vadv(*args(fs3)) == -5


def test_vadv_workspace_bytes(L):
    """c' and, unless it can be parked in the output, a second term per domain point
    (binary64: s = u_stage + u_pos for the y back substitution)."""
    dom = (10, 7, 5)
    n = 10 * 7 * 5
    assert L.vadv_workspace_bytes(2, 0, dom) == 16 * n
    assert L.vadv_workspace_bytes(1, 0, dom) == 4 * n
    assert L.vadv_workspace_bytes(1, 1, dom) == 16 * n
    assert L.vadv_workspace_bytes(1, 2, dom) == 16 * n
    assert L.vadv_workspace_bytes(3, 0, dom) == 0


def test_vadv_workspace_alias_rejected(L):
    G = 1 << 24
    fs = [fake(L, 10, 10, 6, origin=(1, 1, 0), ptr=n * G) for n in range(1, 7)]
    args = [*[ctypes.byref(f) for f in fs], 0.15, 0.0, 0, 0, (ctypes.c_int64 * 3)(8, 8, 6)]
    assert L.lib().gtb_vadv(*args, ctypes.c_void_p(3 * G + 64), 4096, None) == -5
    assert L.lib().gtb_vadv(*args, ctypes.c_void_p(40 * G + 8), 4096, None) == -4  # not 16-byte aligned


def test_hdiff_vadv_validation(L):
    """gtb_hdiff_vadv: in needs the 2-point I/J halo, wcon one point above I, a
    workspace is required, the output may only be utens_stage itself."""
    G = 1 << 24
    fin = lambda o=(2, 2, 0): fake(L, 12, 12, 6, origin=o, ptr=1 * G)
    mk = lambda n, o=(1, 1, 0): fake(L, 10, 10, 6, origin=o, ptr=n * G)
    fs = [fin()] + [mk(n) for n in range(2, 7)]
    lib = L.lib()

    def call(fs, dom=(8, 8, 6), prec=0, flags=0, ws=None, wsb=0):
        d = None if dom is None else (ctypes.c_int64 * 3)(*dom)
        return lib.gtb_hdiff_vadv(*[ctypes.byref(f) for f in fs], 0.15, 0.0, prec, flags, d,
                                  None if ws is None else ctypes.c_void_p(ws), wsb, None)

    assert call(fs, dom=(0, 8, 6)) == 0                        # empty domain: nothing to do
    assert call(fs) == -9                                       # no workspace
    assert call(fs, ws=40 * G, wsb=8 * 8 * 8 * 6 - 8) == -9     # workspace too small
    assert call(fs, ws=40 * G + 8, wsb=1 << 20) == -4           # not 16-byte aligned
    assert call(fs, ws=3 * G + 64, wsb=1 << 20) == -5           # workspace overlaps wcon
    assert call(fs, dom=(9, 8, 6), ws=40 * G, wsb=1 << 20) == -3  # wcon needs i+1 <= 9
    assert call([fin((1, 2, 0))] + fs[1:], ws=40 * G, wsb=1 << 20) == -3  # in needs 2 halo points
    assert call(fs, prec=1, ws=40 * G, wsb=1 << 20) == -9       # FP64 storage: binary64 only
    assert call(fs, flags=2, ws=40 * G, wsb=1 << 20) == -9      # only GTB_WCON_LITERAL
    fs_shift = fs[:5] + [mk(5, o=(1, 2, 0))]                    # output overlapping utens_stage shifted
    assert call(fs_shift, ws=40 * G, wsb=1 << 20) == -5
    fs_in = fs[:5] + [mk(3)]                                    # output on wcon
    assert call(fs_in, ws=40 * G, wsb=1 << 20) == -5
    fs_dt = fs[:3] + [fake(L, 10, 10, 6, origin=(1, 1, 0), dtype=1, ptr=4 * G)] + fs[4:]
    assert call(fs_dt, ws=40 * G, wsb=1 << 20) == -2
    # the deduced domain: min over fields of shape - origin - reach (in: 12-2-2 = 8, wcon: 10-1-1 = 8)
    n = 8 * 8 * 6
    dom = (ctypes.c_int64 * 3)(8, 8, 6)
    assert L.lib().gtb_hdiff_vadv_workspace_bytes(2, 0, 0, dom) == 8 * n       # c' (e parked in the output)
    assert L.lib().gtb_hdiff_vadv_workspace_bytes(2, 0, 4, dom) == 16 * n      # + 1/p (GTB_SAVE_FACTORS)
    # binary32 storage: then h itself, rows padded to 32 values, 256-byte aligned after the state
    h = 4 * 32 * 8 * 6
    up256 = lambda b: (b + 255) // 256 * 256
    assert L.lib().gtb_hdiff_vadv_workspace_bytes(1, 2, 0, dom) == up256(16 * n) + h  # double-float c' and e
    assert L.lib().gtb_hdiff_vadv_workspace_bytes(1, 2, 4, dom) == up256(24 * n) + h
    assert L.lib().gtb_hdiff_vadv_workspace_bytes(1, 0, 4, dom) == up256(8 * n) + h   # binary32 c' and 1/p
    # the workspace with GTB_SAVE_FACTORS must be the larger size
    assert call(fs, flags=4, ws=40 * G, wsb=8 * n) == -9
    # gtb_vadv_adj: GTB_ADJ_FACTORS needs a workspace of the forward's factors
    fw, fy = mk(3), mk(4)
    adj = lambda flags, ws=None, wsb=0: lib.gtb_vadv_adj(ctypes.byref(fw), ctypes.byref(fy), None, None,
                                                         ctypes.byref(mk(5)), None, 0.15, 0.0, 0, flags, dom,
                                                         None if ws is None else ctypes.c_void_p(ws), wsb, None)
    assert adj(8) == -9
    assert adj(8, ws=40 * G, wsb=8 * n) == -9
    assert adj(16) == -9                                                      # unknown flag
    assert adj(8, ws=3 * G, wsb=16 * n) == -5                                 # overlaps wcon


def test_step_validation(L):
    """gtb_step: the checks of gtb_hdiff and gtb_vadv over one shared domain, a
    required workspace, hdiff_out overlapping nothing."""
    G = 1 << 24
    fin = lambda n, o=(2, 2, 0): fake(L, 12, 12, 6, origin=o, ptr=n * G)
    mk = lambda n, o=(1, 1, 0): fake(L, 10, 10, 6, origin=o, ptr=n * G)
    fs = [fin(1), fin(2), fin(3)] + [mk(n) for n in range(4, 10)]
    lib = L.lib()

    def call(fs, dom=(8, 8, 6), prec=0, flags=0, ws=None, wsb=0):
        d = None if dom is None else (ctypes.c_int64 * 3)(*dom)
        return lib.gtb_step(*[ctypes.byref(f) for f in fs], 0.15, 0.0, prec, flags, d,
                            None if ws is None else ctypes.c_void_p(ws), wsb, None)

    ok_ws = dict(ws=40 * G, wsb=1 << 20)
    assert call(fs, dom=(8, 0, 6)) == 0                           # empty domain
    assert call(fs) == -9                                          # workspace required
    assert call(fs, ws=40 * G, wsb=100) == -9                      # too small
    assert call(fs, ws=40 * G + 8, wsb=1 << 20) == -4              # misaligned
    assert call(fs, ws=5 * G, wsb=1 << 20) == -5                   # overlaps wcon
    assert call(fs, dom=(9, 8, 6), **ok_ws) == -3                  # wcon needs i+1
    assert call(fs, prec=2, **ok_ws) == -9                         # FP64 storage: binary64 only
    assert call(fs, flags=8, **ok_ws) == -9
    assert call(fs, flags=16, **ok_ws) == -9                       # GTB_STATE48: FP32 + double-float only
    assert call(fs[:2] + [fin(1)] + fs[3:], **ok_ws) == -5         # hdiff_out on in
    assert call(fs[:2] + [mk(4)] + fs[3:], **ok_ws) == -5          # hdiff_out on u_stage
    assert call(fs[:8] + [mk(6)], **ok_ws) == -5                   # vadv output on u_pos
    assert call(fs[:8] + [fin(3)], **ok_ws) == -5                  # vadv output on hdiff_out
    assert call(fs[:8] + [mk(8, o=(1, 2, 0))], **ok_ws) == -5      # shifted view of utens_stage
    fs_dt = fs[:6] + [fake(L, 10, 10, 6, origin=(1, 1, 0), dtype=1, ptr=7 * G)] + fs[7:]
    assert call(fs_dt, **ok_ws) == -2


def test_selftest_wait_arguments(L):
    """Argument checks run before any launch (no GPU needed)."""
    lib = L.lib()
    for limit, arrive in ((0, 0), (-1, 1), (2_000_000_001, 0), (1000, 3)):
        assert lib.gtb_selftest_wait(limit, arrive, None) == -9


def test_binding_export_list_matches_header(L):
    """The Python binding names every entry point the header declares, and nothing else."""
    assert sorted(L.EXPORTS) == declared_symbols()


def test_fp64_probe_validation(L):
    """The FP64 FMA-rate probe rejects bad sizes and a NULL or misaligned sink before launching."""
    lib = L.lib()
    assert lib.gtb_probe_fp64_fma(0, 16, ctypes.c_void_p(0x10000000), None) == -9
    assert lib.gtb_probe_fp64_fma(8, 0, ctypes.c_void_p(0x10000000), None) == -9
    assert lib.gtb_probe_fp64_fma(8, 16, None, None) == -1
    assert lib.gtb_probe_fp64_fma(8, 16, ctypes.c_void_p(0x10000004), None) == -4
