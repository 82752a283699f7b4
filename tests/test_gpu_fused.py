"""GPU parity of gtb_hdiff_vadv (hdiff feeding vadv in one kernel) against the
oracle composition h = hdiff(in, coeff); utens_stage_out = vadv(h, wcon, h,
utens, utens_stage) (GT4Py paper Sec. 3.1, the two stencils chained).  Bounds
as for the separate stencils: FP64 1e-12 max-norm relative; FP32 storage with
binary64 or double-float column arithmetic 1e-5 against the oracle run in FP64
on the FP32-rounded inputs (the all-binary32 form, which cannot meet that
bound, must be as accurate as the separate chain)."""
import numpy as np
import pytest

from helpers import region, rel_err, s7_stats

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


def draw(I, J, K, seed, wamp=0.5):
    """in, coeff over an (I+4) x (J+4) x K storage (halo 2), the vadv fields over
    (I+2) x (J+2) x K (halo 1), the distributions of the separate stencils."""
    rng = np.random.default_rng(seed)
    hs, vs = (K, J + 4, I + 4), (K, J + 2, I + 2)
    return dict(inp=rng.uniform(-1, 1, hs), coeff=rng.uniform(0, 0.025, hs), wcon=rng.uniform(-wamp, wamp, vs),
                utens=rng.uniform(-1, 1, vs), utens_stage=rng.uniform(-1, 1, vs))


def oracle_chain(orc, f, dom, beta_v=0.0, literal=False):
    I, J, K = dom
    h = region(orc.hdiff(f["inp"], f["coeff"], origin_in=(2, 2, 0), domain=dom), (2, 2, 0), dom)
    hs = np.zeros_like(f["utens"])
    hs[:, 1:1 + J, 1:1 + I] = h
    out = orc.vadv(hs, f["wcon"], hs, f["utens"], f["utens_stage"], origin=(1, 1, 0), domain=dom, beta_v=beta_v,
                   wmode=1 if literal else 0)
    return region(out, (1, 1, 0), dom)


def run_gpu(G, f, dom, dtype=np.float64, prec="native", fused=True, beta_v=0.0, literal=False, inplace=False,
            contiguous=False):
    import torch
    g = {k: v.astype(dtype) for k, v in f.items()}
    if contiguous:  # plain tensors: pitches that are not 16-byte multiples
        sin, scf = (G.Storage(torch.from_numpy(g[k]).cuda(), (2, 2, 0)) for k in ("inp", "coeff"))
    else:
        sin, scf = G.storage_from(g["inp"], (2, 2, 0)), G.storage_from(g["coeff"], (2, 2, 0))
    sv = {k: G.storage_from(g[k], (1, 1, 0)) for k in ("wcon", "utens", "utens_stage")}
    out = sv["utens_stage"] if inplace else G.storage_from(np.zeros_like(g["utens"]), (1, 1, 0))
    if fused:
        G.hdiff_vadv(sin, scf, sv["wcon"], sv["utens"], sv["utens_stage"], out, prec=prec, beta_v=beta_v,
                     literal=literal, domain=dom)
    else:
        h = G.storage_from(np.zeros_like(g["utens"]), (1, 1, 0))
        G.hdiff(sin, scf, h, domain=dom)
        G.vadv(h, sv["wcon"], h, sv["utens"], sv["utens_stage"], out, prec=prec, beta_v=beta_v, literal=literal,
               domain=dom)
    G.device_status()
    return region(out.numpy(), (1, 1, 0), dom)


def test_256_fp64_full_field(G, orc):
    """256x256x80 FP64, the benchmark's launch configuration; whole field."""
    dom = (256, 256, 80)
    f = draw(*dom, 0)
    st = s7_stats(run_gpu(G, f, dom), oracle_chain(orc, f, dom), F64_TOL)
    print("fused chain 256x256x80 FP64:", st)
    assert st["max_norm"] <= F64_TOL
    assert st["p99_9_pointwise"] <= F64_TOL
    assert st["worst_column"] <= 2e-10  # sanity bound, as for gtb_step's column solve


@pytest.mark.parametrize("I,J,K", [(64, 64, 40), (96, 40, 37), (33, 7, 1), (1, 1, 2), (31, 5, 3), (70, 9, 137),
                                   (3, 65, 17), (65, 3, 600)])
def test_shapes_fp64(G, orc, I, J, K):
    """Ragged warps in I, odd J (a half-empty block row), K = 1, 2, 3 and K beyond the
    separate vadv's shared-memory limit (the fused form keeps no column state on chip)."""
    dom = (I, J, K)
    f = draw(*dom, I * J + K, wamp=0.15 if K > 200 else 0.5)
    assert rel_err(run_gpu(G, f, dom), oracle_chain(orc, f, dom)) <= F64_TOL


@pytest.mark.parametrize("beta_v,literal", [(0.3, False), (0.0, True), (-0.2, True)])
def test_beta_and_literal_fp64(G, orc, beta_v, literal):
    dom = (96, 40, 37)
    f = draw(*dom, 5)
    assert rel_err(run_gpu(G, f, dom, beta_v=beta_v, literal=literal),
                   oracle_chain(orc, f, dom, beta_v, literal)) <= F64_TOL


def test_inplace_fp64(G, orc):
    """utens_stage_out on utens_stage itself."""
    dom = (70, 21, 30)
    f = draw(*dom, 6)
    assert rel_err(run_gpu(G, f, dom, inplace=True), oracle_chain(orc, f, dom)) <= F64_TOL


def test_unpadded_in_fp64(G, orc):
    """in and coeff as plain tensors with a pitch of (I+4)*8 bytes, not a 16-byte
    multiple: the producer loads the box itself instead of by TMA."""
    dom = (71, 9, 12)
    f = draw(*dom, 7)
    assert rel_err(run_gpu(G, f, dom, contiguous=True), oracle_chain(orc, f, dom)) <= F64_TOL


def test_matches_unfused_chain_fp64(G, orc):
    """The fused result and gtb_hdiff + gtb_vadv agree to rounding (different order
    of the back substitution, the same unknowns)."""
    dom = (128, 40, 80)
    f = draw(*dom, 8)
    a, b = run_gpu(G, f, dom), run_gpu(G, f, dom, fused=False)
    assert rel_err(a, b) <= 2 * F64_TOL


def test_fp64_tiny_and_nonfinite(G, orc):
    """A level of magnitude 2^-1000 (outside the fixed-point window: the binary64
    definition) and an inf: non-finite columns match the oracle's, the rest within
    the bound."""
    dom = (80, 12, 6)
    f = draw(*dom, 9)
    f["inp"][2] *= 2.0 ** -1000
    f["inp"][4, 7, 40] = np.inf
    got, ref = run_gpu(G, f, dom), oracle_chain(orc, f, dom)
    fin = np.isfinite(ref)
    assert (~fin).sum() > 0
    assert np.array_equal(fin, np.isfinite(got))
    assert rel_err(got[fin], ref[fin]) <= F64_TOL


def test_unread_corners_ignored(G, orc):
    """Arbitrary contents in the halo cells hdiff never reads (three per domain corner):
    a huge finite value and a NaN change nothing, in the fused and the separate hdiff."""
    dom = (40, 12, 3)
    f = draw(*dom, 10)
    ref = oracle_chain(orc, f, dom)
    I, J = dom[0], dom[1]
    for v in (1e300, np.nan):
        g = {k: a.copy() for k, a in f.items()}
        for (ci, cj) in ((-2, -2), (-2, -1), (-1, -2)):
            for (si, sj) in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
                i = ci if si > 0 else I - 1 - ci
                j = cj if sj > 0 else J - 1 - cj
                g["inp"][:, j + 2, i + 2] = v
        assert rel_err(run_gpu(G, g, dom), ref) <= F64_TOL
        sin, scf = G.storage_from(g["inp"], (2, 2, 0)), G.storage_from(g["coeff"], (2, 2, 0))
        sout = G.storage_from(np.zeros_like(g["coeff"]), (2, 2, 0))
        G.hdiff(sin, scf, sout, domain=dom)
        G.device_status()
        href = region(orc.hdiff(f["inp"], f["coeff"], domain=dom), (2, 2, 0), dom)
        assert rel_err(region(sout.numpy(), (2, 2, 0), dom), href) <= F64_TOL


@pytest.mark.parametrize("prec", ["f64", "df"])
@pytest.mark.parametrize("I,J,K", [(96, 40, 37), (256, 256, 80)])
def test_fp32_storage(G, orc, prec, I, J, K):
    """FP32 storage with binary64 / double-float column arithmetic against the oracle
    on the FP32-rounded inputs."""
    dom = (I, J, K)
    f = draw(*dom, 3)
    f32 = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
    assert rel_err(run_gpu(G, f, dom, np.float32, prec), oracle_chain(orc, f32, dom)) <= F32_TOL


@pytest.mark.parametrize("prec", ["native", "f64", "df"])
def test_fp32_chain_equals_separate_calls(G, orc, prec):
    """FP32 storage: gtb_hdiff_vadv runs gtb_hdiff's and gtb_vadv's kernels back to back
    with h in its workspace, so its result equals the two separate calls bit for bit
    (all-binary32, which cannot meet 1e-5 on ill-conditioned columns, included)."""
    dom = (96, 40, 37)
    f = draw(*dom, 4)
    a = run_gpu(G, f, dom, np.float32, prec)
    b = run_gpu(G, f, dom, np.float32, prec, fused=False)
    assert np.array_equal(a, b), prec


def test_workspace_required(G):
    dom = (8, 8, 4)
    f = draw(*dom, 1)
    sin, scf = G.storage_from(f["inp"], (2, 2, 0)), G.storage_from(f["coeff"], (2, 2, 0))
    sv = {k: G.storage_from(f[k], (1, 1, 0)) for k in ("wcon", "utens", "utens_stage")}
    with pytest.raises(G.GtbError) as e:
        G.hdiff_vadv(sin, scf, sv["wcon"], sv["utens"], sv["utens_stage"], workspace=None)
    assert e.value.code == -9


def draw_padded(I, J, K, seed, pad):
    """The same fields with extra storage beyond the halos (origins shifted by pad):
    the TMA box of `in` then starts off the 16-byte boundary for odd i shifts."""
    pi, pj, pk = pad
    rng = np.random.default_rng(seed)
    hs, vs = (K + 2 * pk, J + 4 + 2 * pj, I + 4 + 2 * pi), (K + 2 * pk, J + 2 + 2 * pj, I + 2 + 2 * pi)
    return dict(inp=rng.uniform(-1, 1, hs), coeff=rng.uniform(0, 0.025, hs), wcon=rng.uniform(-0.5, 0.5, vs),
                utens=rng.uniform(-1, 1, vs), utens_stage=rng.uniform(-1, 1, vs))


@pytest.mark.parametrize("pad", [(1, 0, 0), (3, 2, 1), (5, 1, 2)])
def test_origin_offsets_fp64(G, orc, pad):
    I, J, K = 70, 21, 9
    dom = (I, J, K)
    pi, pj, pk = pad
    f = draw_padded(I, J, K, 31, pad)
    oh, ov = (2 + pi, 2 + pj, pk), (1 + pi, 1 + pj, pk)
    sin, scf = G.storage_from(f["inp"], oh), G.storage_from(f["coeff"], oh)
    sv = {k: G.storage_from(f[k], ov) for k in ("wcon", "utens", "utens_stage")}
    out = G.storage_from(np.zeros_like(f["utens"]), ov)
    G.hdiff_vadv(sin, scf, sv["wcon"], sv["utens"], sv["utens_stage"], out, domain=dom)
    G.device_status()
    h = region(orc.hdiff(f["inp"], f["coeff"], origin_in=oh, domain=dom), oh, dom)
    hs = np.zeros_like(f["utens"])
    hs[pk:pk + K, 1 + pj:1 + pj + J, 1 + pi:1 + pi + I] = h
    ref = region(orc.vadv(hs, f["wcon"], hs, f["utens"], f["utens_stage"], origin=ov, domain=dom), ov, dom)
    assert rel_err(region(out.numpy(), ov, dom), ref) <= F64_TOL


@pytest.mark.parametrize("prec", ["native", "f64", "df"])
@pytest.mark.parametrize("I,J,K", [(1, 1, 2), (17, 9, 3), (33, 24, 1)])
def test_small_fp32(G, orc, prec, I, J, K):
    """Ragged FP32 domains (partial tiles and warps, K = 1): the chained call equals the
    two separate calls bit for bit, and meets 1e-5 against the oracle with binary64 or
    double-float columns."""
    dom = (I, J, K)
    f = draw(*dom, 13)
    a = run_gpu(G, f, dom, np.float32, prec)
    b = run_gpu(G, f, dom, np.float32, prec, fused=False)
    f32 = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
    ref = oracle_chain(orc, f32, dom)
    assert np.array_equal(a, b)
    if prec != "native":
        assert rel_err(a, ref) <= F32_TOL
