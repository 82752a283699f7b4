"""GPU parity of gtb_hdiff against the FP64 oracle (GT4Py paper Sec. 3.1,
horizontal diffusion).  FP64 bound: 1e-12 max-norm relative; FP32 bound: 1e-5
against the oracle run in FP64 on the FP32-rounded inputs."""
import numpy as np
import pytest

from helpers import hdiff_point_bound, region, rel_err, s7_stats

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    return gtb


def draw(I, J, K, seed, pad=(0, 0, 0)):
    """in and coeff over an (I+4+2*pad_i) x (J+4+2*pad_j) x (K+2*pad_k) storage."""
    rng = np.random.default_rng(seed)
    shp = (K + 2 * pad[2], J + 4 + 2 * pad[1], I + 4 + 2 * pad[0])
    return rng.uniform(-1, 1, shp), rng.uniform(0, 0.025, shp)


def run_case(G, orc, I, J, K, seed=0, dtype=np.float64, pad=(0, 0, 0), contiguous=False):
    import torch
    inp, coeff = draw(I, J, K, seed, pad)
    if dtype == np.float32:
        inp, coeff = inp.astype(np.float32), coeff.astype(np.float32)
    o = (2 + pad[0], 2 + pad[1], pad[2])
    dom = (I, J, K)
    if contiguous:   # plain torch tensors: unpadded rows, odd pitches
        tin = torch.from_numpy(inp).cuda()
        tcf = torch.from_numpy(coeff).cuda()
        tout = torch.zeros_like(tcf)
        sin, scf, sout = G.Storage(tin, o), G.Storage(tcf, o), G.Storage(tout, o)
    else:
        sin, scf = G.storage_from(inp, o), G.storage_from(coeff, o)
        sout = G.storage_from(np.zeros_like(coeff), o)
    G.hdiff(sin, scf, sout, domain=dom)
    G.device_status()
    got = region(sout.numpy(), o, dom)
    ref = region(orc.hdiff(inp.astype(np.float64), coeff.astype(np.float64), origin_in=o, domain=dom), o, dom)
    return got, ref


def test_small_fp64(G, orc):
    """64x64x40, halo 2 (storage 68x68x40), in ~ U(-1,1), coeff ~ U(0,0.025), seed 0."""
    got, ref = run_case(G, orc, 64, 64, 40)
    assert rel_err(got, ref) <= F64_TOL


def test_256_fp64_full_field(G, orc):
    """256x256x80 FP64, the launch configuration the benchmark times; whole field.
    Beside the max-norm: the per-point bound of the fixed-point form, the worst column,
    the 99.9th percentile of the pointwise error and the fraction of points beyond 1e-12."""
    got, ref = run_case(G, orc, 256, 256, 80, seed=1)
    inp, coeff = draw(256, 256, 80, 1)
    st = s7_stats(got, ref, F64_TOL)
    print("hdiff 256x256x80 FP64:", st)
    assert st["max_norm"] <= F64_TOL
    assert np.all(np.abs(got - ref) <= hdiff_point_bound(ref, inp, coeff, (2, 2, 0), (256, 256, 80)))
    assert st["worst_column"] <= F64_TOL
    assert st["p99_9_pointwise"] <= F64_TOL


@pytest.mark.parametrize("I,J,K", [(67, 19, 5), (1, 1, 1), (130, 3, 2), (65, 17, 1), (200, 33, 7), (63, 15, 3)])
def test_ragged_fp64(G, orc, I, J, K):
    """Domains that leave ragged tiles in I and J, one-point and one-level domains."""
    got, ref = run_case(G, orc, I, J, K, seed=I + J + K)
    assert rel_err(got, ref) <= F64_TOL


@pytest.mark.parametrize("pad", [(1, 0, 0), (3, 2, 1), (5, 1, 2)])
def test_origin_offsets_fp64(G, orc, pad):
    """Non-zero origins beyond the halo, including odd i origins (TMA box shifted
    to the 16-byte boundary)."""
    got, ref = run_case(G, orc, 70, 21, 6, seed=3, pad=pad)
    assert rel_err(got, ref) <= F64_TOL


@pytest.mark.parametrize("I,J", [(71, 9), (64, 16)])
def test_unpadded_layouts(G, orc, I, J):
    """Plain contiguous tensors: pitches that are not 16-byte multiples take the
    cooperative-load path and scalar stores."""
    for dt in (np.float64, np.float32):
        got, ref = run_case(G, orc, I, J, 4, seed=7, dtype=dt, contiguous=True)
        assert rel_err(got, ref) <= (F64_TOL if dt == np.float64 else F32_TOL)


def test_fp32_512(G, orc):
    """512x512x80 with FP32 storage and arithmetic (the precision form)."""
    got, ref = run_case(G, orc, 512, 512, 80, seed=0, dtype=np.float32)
    assert rel_err(got, ref) <= F32_TOL


@pytest.mark.parametrize("I,J,K", [(129, 17, 3), (5, 300, 2)])
def test_ragged_fp32(G, orc, I, J, K):
    got, ref = run_case(G, orc, I, J, K, seed=11, dtype=np.float32)
    assert rel_err(got, ref) <= F32_TOL


def test_closed_forms_on_gpu(G, orc):
    """The oracle's closed forms hold on the GPU too: constant and quartic fields."""
    import torch
    I, J, K = 40, 24, 3
    k, y, x = np.meshgrid(np.arange(K), np.arange(J + 4), np.arange(I + 4), indexing="ij")
    coeff = np.random.default_rng(5).integers(0, 26, x.shape) / 1024.0
    for inp, expect in ((np.full(x.shape, 0.375), lambda a: a), (((x - 20.0) ** 4), lambda a: a + 24.0 * coeff)):
        sin, scf = G.storage_from(inp, (2, 2, 0)), G.storage_from(coeff, (2, 2, 0))
        sout = G.storage_from(np.zeros_like(coeff), (2, 2, 0))
        G.hdiff(sin, scf, sout)
        got = region(sout.numpy(), (2, 2, 0), (I, J, K))
        assert np.array_equal(got, region(expect(inp), (2, 2, 0), (I, J, K)))


def test_out_of_range_errors_on_gpu(G):
    import torch
    a = G.storage_from(np.zeros((2, 8, 8)), (2, 2, 0))
    b = G.storage_from(np.zeros((2, 8, 8)), (2, 2, 0))
    with pytest.raises(G.GtbError) as e:
        G.hdiff(a, b, a)
    assert e.value.code == -5
    with pytest.raises(G.GtbError) as e:
        G.hdiff(a, b, G.storage_from(np.zeros((2, 8, 8)), (2, 2, 0)), domain=(5, 4, 2))
    assert e.value.code == -3


def run_fields(G, orc, inp, coeff, origin=(2, 2, 0)):
    nk, nj, ni = inp.shape
    dom = (ni - 4, nj - 4, nk)
    sin, scf = G.storage_from(inp, origin), G.storage_from(coeff, origin)
    sout = G.storage_from(np.zeros_like(coeff), origin)
    G.hdiff(sin, scf, sout)
    G.device_status()
    return region(sout.numpy(), origin, dom), region(orc.hdiff(inp, coeff), origin, dom)


def test_fp64_nonfinite_tile_takes_binary64_phases(G, orc):
    """An inf in one tile: that tile level runs the binary64 phases, every other tile
    the fixed-point form; non-finite outputs and finite values match the oracle."""
    inp, coeff = draw(150, 40, 3, 21)
    inp[1, 12, 30] = np.inf
    inp[2, 30, 100] = np.nan
    got, ref = run_fields(G, orc, inp, coeff)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    assert (~fin).sum() > 0
    assert rel_err(got[fin], ref[fin]) <= F64_TOL


def test_fp64_tiny_magnitudes(G, orc):
    """A field of magnitude 2^-1000 (exponents outside the fixed-point window)."""
    inp, coeff = draw(70, 20, 2, 22)
    got, ref = run_fields(G, orc, inp * 2.0 ** -1000, coeff)
    assert rel_err(got, ref) <= F64_TOL


def test_fp64_wide_dynamic_range(G, orc):
    """Inputs spanning 60 binades in every tile: small values are truncated in the
    fixed-point form, far below the bound relative to the field maximum.  The error is
    absolute at the level's scale: every point meets the per-point bound, while points
    far below the tile's largest input keep fewer significant bits than binary64 (their
    pointwise relative error is reported, not bounded by 1e-12)."""
    inp, coeff = draw(130, 33, 4, 23)
    scale = 2.0 ** np.random.default_rng(24).integers(-60, 1, inp.shape)
    got, ref = run_fields(G, orc, inp * scale, coeff)
    st = s7_stats(got, ref, F64_TOL)
    print("hdiff wide dynamic range FP64:", st)
    assert st["max_norm"] <= F64_TOL
    assert np.all(np.abs(got - ref) <= hdiff_point_bound(ref, inp * scale, coeff, (2, 2, 0), (130, 33, 4)))


def test_fp64_limiter_sign_of_tiny_differences(G, orc):
    """Neighbours that differ only in their last bit, far below the fixed-point
    resolution of their tile: the limiter still sees the exact sign of in[i+1]-in[i]."""
    inp, coeff = draw(64, 16, 2, 25)
    x0 = 1e-200
    x1 = np.nextafter(x0, 1.0)
    inp[:, 8:12, 20] = x0
    inp[:, 8:12, 21] = x1
    inp[:, 8:12, 22] = x0
    got, ref = run_fields(G, orc, inp, coeff)
    assert rel_err(got, ref) <= F64_TOL
