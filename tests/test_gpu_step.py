"""GPU parity of gtb_step: the benchmark's two stencils on their own fields in
one co-scheduled kernel (GT4Py paper Sec. 3.1).  hdiff_out against the FP64
oracle (1e-12 max-norm relative; FP32 storage 1e-5 on the FP32-rounded
inputs); utens_stage_out against gtb_vadv with the same workspace form, bit
for bit (the same column code), and through it against the oracle."""
import numpy as np
import pytest

from helpers import hdiff_point_bound, region, rel_err, s7_stats

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5
VN = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")
# The column solve's worst column has no a-priori bound: it scales with the column's
# conditioning.  On these draws (256x256x80, seed 0) the binary64 oracle itself is
# 2.7e-11 from an extended-precision Thomas solve in its worst column (max-norm 2.5e-13,
# 99.9th percentile 4.1e-14): a sanity bound about 7x above that.
VADV_WORST_COLUMN = 2e-10


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    return gtb


def draw(I, J, K, seed, wamp=0.5):
    rng = np.random.default_rng(seed)
    hs, vs = (K, J + 4, I + 4), (K, J + 2, I + 2)
    f = dict(inp=rng.uniform(-1, 1, hs), coeff=rng.uniform(0, 0.025, hs))
    for n in ("u_stage", "u_pos", "utens", "utens_stage"):
        f[n] = rng.uniform(-1, 1, vs)
    f["wcon"] = rng.uniform(-wamp, wamp, vs)
    return f


def run(G, f, dom, dtype=np.float64, prec="native", beta_v=0.0, literal=False, inplace=False, contiguous=False,
        state48=False):
    """(hdiff_out, utens_stage_out) of gtb_step, and utens_stage_out of gtb_vadv."""
    import torch
    g = {k: v.astype(dtype) for k, v in f.items()}
    if contiguous:
        sin, scf = (G.Storage(torch.from_numpy(g[k]).cuda(), (2, 2, 0)) for k in ("inp", "coeff"))
    else:
        sin, scf = G.storage_from(g["inp"], (2, 2, 0)), G.storage_from(g["coeff"], (2, 2, 0))
    hout = G.storage_from(np.zeros_like(g["coeff"]), (2, 2, 0))
    sv = {n: G.storage_from(g[n], (1, 1, 0)) for n in VN}
    vout = sv["utens_stage"] if inplace else G.storage_from(np.zeros_like(g["utens"]), (1, 1, 0))
    kw = dict(prec=prec, beta_v=beta_v, literal=literal, domain=dom, state48=state48)
    ref_v = G.storage_from(np.zeros_like(g["utens"]), (1, 1, 0))
    G.vadv(*[sv[n] for n in VN], ref_v, **kw)  # before an in-place step overwrites utens_stage
    G.step(sin, scf, hout, *[sv[n] for n in VN], vout, **kw)
    G.device_status()
    return (region(hout.numpy(), (2, 2, 0), dom), region(vout.numpy(), (1, 1, 0), dom),
            region(ref_v.numpy(), (1, 1, 0), dom))


def oracle(orc, f, dom, beta_v=0.0, literal=False):
    h = region(orc.hdiff(f["inp"], f["coeff"], origin_in=(2, 2, 0), domain=dom), (2, 2, 0), dom)
    v = region(orc.vadv(*[f[n] for n in VN], origin=(1, 1, 0), domain=dom, beta_v=beta_v,
                        wmode=1 if literal else 0), (1, 1, 0), dom)
    return h, v


def test_256_fp64_full_field(G, orc):
    """256x256x80 FP64, the benchmark's workload and launch configuration."""
    dom = (256, 256, 80)
    f = draw(*dom, 0)
    h, v, v1 = run(G, f, dom)
    rh, rv = oracle(orc, f, dom)
    sh, sv = s7_stats(h, rh, F64_TOL), s7_stats(v, rv, F64_TOL)
    print("step 256x256x80 FP64 hdiff_out:", sh)
    print("step 256x256x80 FP64 utens_stage_out:", sv)
    assert sh["max_norm"] <= F64_TOL
    assert np.all(np.abs(h - rh) <= hdiff_point_bound(rh, f["inp"], f["coeff"], (2, 2, 0), dom))
    assert sh["worst_column"] <= F64_TOL and sh["p99_9_pointwise"] <= F64_TOL
    assert np.array_equal(v, v1)
    assert sv["max_norm"] <= F64_TOL
    assert sv["p99_9_pointwise"] <= F64_TOL
    assert sv["worst_column"] <= VADV_WORST_COLUMN


@pytest.mark.parametrize("I,J,K", [(64, 64, 40), (96, 40, 37), (33, 7, 1), (1, 1, 2), (31, 5, 3), (70, 9, 137),
                                   (3, 65, 17)])
def test_shapes_fp64(G, orc, I, J, K):
    dom = (I, J, K)
    f = draw(*dom, I * J + K)
    h, v, v1 = run(G, f, dom)
    rh, rv = oracle(orc, f, dom)
    assert rel_err(h, rh) <= F64_TOL
    assert np.array_equal(v, v1)
    assert rel_err(v, rv) <= F64_TOL


@pytest.mark.parametrize("beta_v,literal,inplace", [(0.3, False, False), (0.0, True, True), (-0.2, True, False)])
def test_options_fp64(G, orc, beta_v, literal, inplace):
    dom = (96, 40, 37)
    f = draw(*dom, 5)
    h, v, v1 = run(G, f, dom, beta_v=beta_v, literal=literal, inplace=inplace)
    rh, rv = oracle(orc, f, dom, beta_v, literal)
    assert rel_err(h, rh) <= F64_TOL
    assert np.array_equal(v, v1)
    assert rel_err(v, rv) <= F64_TOL


def test_unpadded_in_fp64(G, orc):
    """in as a plain tensor (pitch not a 16-byte multiple): no TMA, producer loads."""
    dom = (71, 9, 12)
    f = draw(*dom, 7)
    h, v, v1 = run(G, f, dom, contiguous=True)
    rh, rv = oracle(orc, f, dom)
    assert rel_err(h, rh) <= F64_TOL and np.array_equal(v, v1)


def test_unread_corners_and_nonfinite_fp64(G, orc):
    """Arbitrary values in the unread halo corners change nothing; an inf in a read
    cell gives the oracle's non-finite pattern."""
    dom = (40, 12, 3)
    f = draw(*dom, 10)
    I, J = dom[0], dom[1]
    for (ci, cj) in ((-2, -2), (-2, -1), (-1, -2)):
        for (si, sj) in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
            i = ci if si > 0 else I - 1 - ci
            j = cj if sj > 0 else J - 1 - cj
            f["inp"][:, j + 2, i + 2] = 1e300
    f["inp"][1, 7, 20] = np.inf
    h, v, v1 = run(G, f, dom)
    rh, _ = oracle(orc, f, dom)
    fin = np.isfinite(rh)
    assert (~fin).sum() > 0 and np.array_equal(fin, np.isfinite(h))
    assert rel_err(h[fin], rh[fin]) <= F64_TOL
    assert np.array_equal(v, v1)


@pytest.mark.parametrize("prec", ["native", "f64", "df", "df48"])
def test_fp32_storage(G, orc, prec):
    """FP32 storage: hdiff_out within 1e-5 of the oracle, utens_stage_out gtb_vadv's bit for
    bit (df48: double-float with the column state in 48 bits, GTB_STATE48, in both calls)."""
    dom = (96, 40, 37)
    f = draw(*dom, 3)
    h, v, v1 = run(G, f, dom, np.float32, prec[:2] if prec == "df48" else prec, state48=prec == "df48")
    f32 = {k: a.astype(np.float32).astype(np.float64) for k, a in f.items()}
    rh, rv = oracle(orc, f32, dom)
    assert rel_err(h, rh) <= F32_TOL
    assert np.array_equal(v, v1)
    if prec != "native":
        assert rel_err(v, rv) <= F32_TOL


def test_workspace_required(G):
    dom = (8, 8, 4)
    f = draw(*dom, 1)
    sin, scf = G.storage_from(f["inp"], (2, 2, 0)), G.storage_from(f["coeff"], (2, 2, 0))
    hout = G.storage_from(np.zeros_like(f["coeff"]), (2, 2, 0))
    sv = {n: G.storage_from(f[n], (1, 1, 0)) for n in VN}
    with pytest.raises(G.GtbError) as e:
        G.step(sin, scf, hout, *[sv[n] for n in VN], workspace=None)
    assert e.value.code == -9


@pytest.mark.parametrize("pad", [(1, 0, 0), (3, 2, 1)])
def test_origin_offsets_fp64(G, orc, pad):
    """Origins beyond the halos (the TMA box of `in` off the 16-byte boundary)."""
    I, J, K = 70, 21, 9
    dom = (I, J, K)
    pi, pj, pk = pad
    rng = np.random.default_rng(41)
    hs, vs = (K + 2 * pk, J + 4 + 2 * pj, I + 4 + 2 * pi), (K + 2 * pk, J + 2 + 2 * pj, I + 2 + 2 * pi)
    f = dict(inp=rng.uniform(-1, 1, hs), coeff=rng.uniform(0, 0.025, hs))
    for n in ("u_stage", "u_pos", "utens", "utens_stage"):
        f[n] = rng.uniform(-1, 1, vs)
    f["wcon"] = rng.uniform(-0.5, 0.5, vs)
    oh, ov = (2 + pi, 2 + pj, pk), (1 + pi, 1 + pj, pk)
    sin, scf = G.storage_from(f["inp"], oh), G.storage_from(f["coeff"], oh)
    hout = G.storage_from(np.zeros_like(f["coeff"]), oh)
    sv = {n: G.storage_from(f[n], ov) for n in VN}
    vout = G.storage_from(np.zeros_like(f["utens"]), ov)
    G.step(sin, scf, hout, *[sv[n] for n in VN], vout, domain=dom)
    G.device_status()
    rh = region(orc.hdiff(f["inp"], f["coeff"], origin_in=oh, domain=dom), oh, dom)
    rv = region(orc.vadv(*[f[n] for n in VN], origin=ov, domain=dom), ov, dom)
    assert rel_err(region(hout.numpy(), oh, dom), rh) <= F64_TOL
    assert rel_err(region(vout.numpy(), ov, dom), rv) <= F64_TOL


@pytest.mark.parametrize("I,J", [(40, 30), (256, 240)])
def test_update_paths_fp64(G, orc, I, J):
    """Every branch of the producers' update out = in - coeff D, in both forms: a
    small grid keeps the binary64 FMA, 256 x 240 (960 CTAs, over 85% of what the GPU
    holds at once) takes the integer pipe.  coeff rows of 0, negative, subnormal,
    normal and >= 1 (the binary64 fallback); levels of ordinary values, huge values (the fallback for a
    large fixed-point scale), small values (fixed point at a small scale; 1e-140, so
    that the oracle's binary64 limiter product cannot underflow: below about 1e-154
    it can, and then it keeps fluxes that the exact sign test limits) and a constant
    (D = 0: out equals in exactly).  Each level against the oracle, relative to its
    own size."""
    K = 4
    dom = (I, J, K)
    f = draw(*dom, 17)
    cf = f["coeff"]
    cf[:, 2:8, :] = 0.0
    cf[:, 8:13, :] = -cf[:, 8:13, :]
    cf[:, 13:17, :] = 3e-310
    cf[:, 28:32, :] = 1.5
    f["inp"][1] *= 1e295
    f["inp"][2] *= 1e-140
    f["inp"][3] = 0.625
    h, _, _ = run(G, f, dom)
    rh, _ = oracle(orc, f, dom)
    for k in range(3):
        assert rel_err(h[k], rh[k]) <= F64_TOL, k
    assert np.array_equal(h[3], np.full_like(h[3], 0.625))


def test_cuda_graph_capture_fp64(G):
    """gtb_step and gtb_hdiff_vadv inside a user's CUDA graph (torch.cuda.graph): after
    one eager call per entry point (the workspace cache and the per-kernel set-up are
    warm), a captured replay enqueues nothing on the host and gives the eager results
    bit for bit, on inputs changed in place between replays."""
    import torch
    dom = (256, 240, 12)
    f = draw(*dom, 23)
    sin, scf = G.storage_from(f["inp"], (2, 2, 0)), G.storage_from(f["coeff"], (2, 2, 0))
    hout = G.storage_from(np.zeros_like(f["coeff"]), (2, 2, 0))
    sv = {n: G.storage_from(f[n], (1, 1, 0)) for n in VN}
    vout = G.storage_from(np.zeros_like(f["utens"]), (1, 1, 0))
    cout = G.storage_from(np.zeros_like(f["utens"]), (1, 1, 0))
    s = torch.cuda.Stream()

    def calls():
        G.step(sin, scf, hout, *[sv[n] for n in VN], vout, domain=dom, stream=s)
        G.hdiff_vadv(sin, scf, sv["wcon"], sv["utens"], sv["utens_stage"], cout, domain=dom, stream=s)

    with torch.cuda.stream(s):
        calls()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        calls()
    for rep in range(2):
        # new inputs in place, then replay against eager calls on the same inputs
        sin.data.mul_(0.5 + rep)
        sv["utens"].data.add_(0.25)
        for st in (hout, vout, cout):
            st.data.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        G.device_status()
        got = [st.numpy().copy() for st in (hout, vout, cout)]
        with torch.cuda.stream(s):
            calls()
        torch.cuda.synchronize()
        for a, st in zip(got, (hout, vout, cout)):
            assert np.array_equal(a, st.numpy(), equal_nan=True)  # halos stay NaN in both
        assert np.isfinite(region(got[0], (2, 2, 0), dom)).all()
        assert np.isfinite(region(got[2], (1, 1, 0), dom)).all()


def test_state48_rejected_fp64(G):
    """GTB_STATE48 applies to FP32 storage with double-float columns only (GTB_ERR_ARG)."""
    dom = (8, 8, 4)
    f = draw(*dom, 1)
    sin, scf = G.storage_from(f["inp"], (2, 2, 0)), G.storage_from(f["coeff"], (2, 2, 0))
    hout = G.storage_from(np.zeros_like(f["coeff"]), (2, 2, 0))
    sv = {n: G.storage_from(f[n], (1, 1, 0)) for n in VN}
    with pytest.raises(G.GtbError) as e:
        G.step(sin, scf, hout, *[sv[n] for n in VN], state48=True)
    assert e.value.code == -9
