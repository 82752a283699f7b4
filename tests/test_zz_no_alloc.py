"""gtb_vadv_noalloc: vadv for callers that cannot allocate device memory.

Some callers run inside a host application that owns every device allocation
(or must not pay cudaMalloc's implicit synchronisation in a time loop), so
they cannot hand gtb_vadv a workspace.  gtb_vadv_noalloc keeps the forward
sweep's state in a fixed array inside the library instead.  These tests call
it through the C ABI and check it against gtb_vadv (the workspace entry
point) on two calls in a row, with different inputs, so that state left in
the shared array by the first call cannot hide an error in the second.  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from helpers import region, rel_err

pytestmark = pytest.mark.gpu

NAMES = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")
F64_TOL = 1e-12
F32_TOL = 1e-5


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    L = gtb.lib()
    P = ctypes.POINTER(gtb.GtbField)
    L.gtb_vadv_noalloc.argtypes = [P, P, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_uint, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    L.gtb_vadv_noalloc.restype = ctypes.c_int
    return gtb


def fields(G, I, J, K, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    shp = (K, J + 2, I + 2)
    f = {n: rng.uniform(-1, 1, shp) for n in ("u_stage", "u_pos", "utens", "utens_stage")}
    f["wcon"] = rng.uniform(-0.5, 0.5, shp)
    return {n: G.storage_from(v.astype(dtype), (1, 1, 0)) for n, v in f.items()}


def call_noalloc(G, st, out, prec=0, domain=None):
    fs = [G.field(st[n]) for n in NAMES] + [G.field(out)]
    dom = None if domain is None else (ctypes.c_int64 * 3)(*domain)
    import torch
    return G.lib().gtb_vadv_noalloc(*[ctypes.byref(f) for f in fs], 0.15, 0.0, prec, 0, dom,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


# the deduced domain reaches one row into the halo (J + 1); 128 x 113 x 64 binary64 needs
# 14.8 MB of the 16 MiB array (two values per point)
@pytest.mark.parametrize("dtype,prec,shape", [(np.float64, "native", (128, 112, 64)),
                                              (np.float32, "df", (100, 70, 80))])
def test_matches_workspace_entry_point_twice(G, dtype, prec, shape):
    I, J, K = shape
    tol = F64_TOL if dtype == np.float64 else F32_TOL
    pcode = G.PREC[prec]
    for seed in (11, 12):  # two calls in a row on different inputs
        st = fields(G, I, J, K, seed, dtype)
        ref = G.storage_from(np.zeros(st["utens"].shape, dtype), (1, 1, 0))
        got = G.storage_from(np.full(st["utens"].shape, np.nan, dtype), (1, 1, 0))
        G.vadv(*[st[n] for n in NAMES], ref, prec=prec)
        rc = call_noalloc(G, st, got, prec=pcode)
        assert rc == 0, G.lib().gtb_last_error().decode()
        G.device_status()
        a = region(got.numpy(), (1, 1, 0), (I, J, K))
        b = region(ref.numpy(), (1, 1, 0), (I, J, K))
        assert np.all(np.isfinite(a))
        assert rel_err(a, b) <= tol, seed


def test_rejects_domains_beyond_the_fixed_array(G):
    st = fields(G, 8, 4, 3, 13)
    out = G.storage_from(np.zeros(st["utens"].shape), (1, 1, 0))
    # 256 x 256 x 80 binary64 needs 80 MiB of scratch; only the domain is checked
    rc = call_noalloc(G, st, out, domain=(256, 256, 80))
    assert rc == -8
    assert "16777216" in G.lib().gtb_last_error().decode()
