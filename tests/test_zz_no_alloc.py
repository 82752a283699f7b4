"""gtb_vadv_noalloc: vadv for callers that cannot allocate device memory.

Some callers run inside a host application that owns every device allocation
(or must not pay cudaMalloc's implicit synchronisation in a time loop), so
they cannot hand gtb_vadv a workspace.  gtb_vadv_noalloc keeps the forward
sweep's state in a fixed array inside the library instead.  These tests call
it through the C ABI on two calls in a row, with different inputs, so that
state left in the shared array by the first call cannot hide an error in the
second, and check each result three ways:

* bit for bit against gtb_vadv with a caller workspace (the same kernel on
  the same arithmetic; only where the state lives differs);
* against the FP64 oracle (1e-12 for binary64 storage, 1e-5 for binary32
  storage with double-float or binary64 columns);
* with an explicit domain smaller than the deduced one, every cell outside it
  keeps what it held before the call.

This file is collected last on purpose."""
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


def draws(I, J, K, seed):
    """Seeded FP64 draws over the storage (halo 1 in I and J) with the benchmark's distributions."""
    rng = np.random.default_rng(seed)
    shp = (K, J + 2, I + 2)
    f = {n: rng.uniform(-1, 1, shp) for n in ("u_stage", "u_pos", "utens", "utens_stage")}
    f["wcon"] = rng.uniform(-0.5, 0.5, shp)
    return f


def upload(G, f, dtype):
    return {n: G.storage_from(v.astype(dtype), (1, 1, 0)) for n, v in f.items()}


def call_noalloc(G, st, out, prec=0, domain=None):
    import torch
    fs = [G.field(st[n]) for n in NAMES] + [G.field(out)]
    dom = None if domain is None else (ctypes.c_int64 * 3)(*domain)
    return G.lib().gtb_vadv_noalloc(*[ctypes.byref(f) for f in fs], 0.15, 0.0, prec, 0, dom,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


# The deduced domain reaches one row into the halo (J + 1 rows): 128 x 113 x 64 binary64
# needs 14.8 MB of the 16 MiB array (two values per point).
@pytest.mark.parametrize("dtype,prec,shape", [(np.float64, "native", (128, 112, 64)),
                                              (np.float32, "df", (100, 70, 80)),
                                              (np.float32, "f64", (64, 40, 33)),
                                              (np.float32, "native", (96, 50, 80))])
def test_matches_workspace_entry_point_and_oracle_twice(G, orc, dtype, prec, shape):
    I, J, K = shape
    dom = (I, J + 1, K)
    pcode = G.PREC[prec]
    for seed in (11, 12):  # two calls in a row on different inputs
        f = draws(I, J, K, seed)
        st = upload(G, f, dtype)
        ref = G.storage_from(np.zeros(f["utens"].shape, dtype), (1, 1, 0))
        got = G.storage_from(np.full(f["utens"].shape, np.nan, dtype), (1, 1, 0))
        G.vadv(*[st[n] for n in NAMES], ref, prec=prec, workspace="auto")
        rc = call_noalloc(G, st, got, prec=pcode)
        assert rc == 0, G.lib().gtb_last_error().decode()
        G.device_status()
        a = region(got.numpy(), (1, 1, 0), dom)
        b = region(ref.numpy(), (1, 1, 0), dom)
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b), seed
        if prec == "native" and dtype == np.float32:
            continue  # binary32 columns do not meet 1e-5 on ill-conditioned columns (by design)
        f64 = {n: v.astype(dtype).astype(np.float64) for n, v in f.items()}
        oracle_out = orc.vadv(*[f64[n] for n in NAMES], domain=dom)
        tol = F64_TOL if dtype == np.float64 else F32_TOL
        assert rel_err(a, region(oracle_out, (1, 1, 0), dom)) <= tol, seed


def test_explicit_domain_leaves_the_rest_untouched(G, orc):
    """An explicit domain inside the deduced one (and one outside the fixed array's
    reach when deduced) writes only its own cells; the rest keeps the sentinel."""
    I, J, K = 200, 120, 60  # deduced 200 x 121 x 60 binary64: 23 MB, above the array
    sub = (136, 90, 48)
    f = draws(I, J, K, 14)
    st = upload(G, f, np.float64)
    sentinel = np.full(f["utens"].shape, 7.25)
    got = G.storage_from(sentinel, (1, 1, 0))
    assert call_noalloc(G, st, got) == -8  # the deduced domain does not fit
    rc = call_noalloc(G, st, got, domain=sub)
    assert rc == 0, G.lib().gtb_last_error().decode()
    G.device_status()
    out = got.numpy()
    ref = orc.vadv(*[f[n] for n in NAMES], domain=sub)
    assert rel_err(region(out, (1, 1, 0), sub), region(ref, (1, 1, 0), sub)) <= F64_TOL
    mask = np.ones(out.shape, bool)
    mask[0:sub[2], 1:1 + sub[1], 1:1 + sub[0]] = False
    assert np.all(out[mask] == 7.25)
    # the same sub-domain again through the workspace entry point: bit for bit
    ref_ws = G.storage_from(sentinel, (1, 1, 0))
    G.vadv(*[st[n] for n in NAMES], ref_ws, domain=sub, workspace="auto")
    G.device_status()
    assert np.array_equal(ref_ws.numpy(), out)


def test_rejects_domains_beyond_the_fixed_array(G):
    st = upload(G, draws(8, 4, 3, 13), np.float64)
    out = G.storage_from(np.zeros(st["utens"].shape), (1, 1, 0))
    # 256 x 256 x 80 binary64 needs 80 MiB of scratch; only the domain is checked
    rc = call_noalloc(G, st, out, domain=(256, 256, 80))
    assert rc == -8
    assert "16777216" in G.lib().gtb_last_error().decode()
