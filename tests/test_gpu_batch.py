"""GPU tests of the batched form: an ensemble of uneven domains run by two
persistent kernels replayed from a CUDA graph (gtb_batch_plan / gtb_batch_run).
Each member computes h = hdiff(in, coeff), out = vadv(h, wcon, h, utens,
utens_stage).  Results must equal the single-domain entry points bit for bit
(same per-point arithmetic) and the oracle composition (the oracle's hdiff
feeding the oracle's vadv) within the bounds: 1e-5 for FP32 storage with
double-float columns, 1e-12 for FP64."""
import numpy as np
import pytest

from helpers import region, rel_err, s7_stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    return gtb


def ensemble(G, n, dtype, seed=0, shapes=None):
    from paper_2311_08322_b300 import inputs
    shapes = shapes or inputs.ensemble_shapes(48, seed)[:n]
    mems = []
    for q, (I, J, K) in enumerate(shapes):
        f = inputs.hdiff_vadv(I, J, K, seed=100 + q, wcon_amp=0.5)
        f = {k: v.astype(dtype) for k, v in f.items()}
        mems.append((G.member_storages(f, I, J, K), f))
    return mems


SHAPES = [(48, 48, 40), (384, 384, 137), (96, 96, 60), (128, 128, 80), (192, 192, 40), (256, 256, 137),
          (48, 48, 137), (96, 96, 40)]


@pytest.mark.parametrize("dtype,prec", [(np.float32, "df"), (np.float64, "native"), (np.float32, "native")])
def test_batch_equals_single_launches(G, dtype, prec):
    mems = ensemble(G, len(SHAPES), dtype, shapes=SHAPES)
    plan = G.BatchPlan([m for m, _ in mems], prec=prec)
    plan.run()
    G.device_status()
    info = plan.info()
    assert info["members"] == len(SHAPES) and info["points"] == sum(I * J * K for I, J, K in SHAPES)
    for m, f in mems:
        I, J, K = m["domain"]
        hb, ob = m["h"].numpy(), region(m["out"].numpy(), (1, 1, 0), (I, J, K))
        single = G.member_storages(f, I, J, K)
        G.run_member_single(single, prec=prec)
        G.device_status()
        assert np.array_equal(hb, single["h"].numpy()), (I, J, K)
        assert np.array_equal(ob, region(single["out"].numpy(), (1, 1, 0), (I, J, K))), (I, J, K)
    plan.close()


def member_draws(I, J, K, q, dtype):
    """Member q of the seed-0 ensemble: its own generator (seed 1 + q), rounded to dtype."""
    from paper_2311_08322_b300 import inputs
    return {k: v.astype(dtype) for k, v in inputs.hdiff_vadv(I, J, K, seed=1 + q).items()}


def oracle_member(orc, f):
    """The oracle composition of one member: h = hdiff(in, coeff) by the oracle, then the
    oracle's vadv on the oracle's own h (u_stage = u_pos = h), in binary64 on the member's
    (possibly FP32-rounded) inputs."""
    f64 = {k: v.astype(np.float64) for k, v in f.items()}
    h = orc.hdiff(f64["in"], f64["coeff"])[:, 2:-2, 2:-2]
    hp = np.pad(h, ((0, 0), (1, 1), (1, 1)))
    out = orc.vadv(hp, f64["wcon"], hp, f64["utens"], f64["utens_stage"])[:, 1:-1, 1:-1]
    return h, out


def extended_member(orc, f, h):
    """The member's vadv output from the oracle's system (its own h as u_stage and u_pos)
    solved column by column by the oracle's extended-precision (x87 long double) Thomas
    recurrences: the reference for how far the binary64 oracle itself is from the
    exact solution on ill-conditioned columns."""
    f64 = {k: v.astype(np.float64) for k, v in f.items()}
    K, J, I = h.shape
    hp = np.pad(h, ((0, 0), (1, 1), (1, 1)))
    out = np.empty_like(h)
    for j in range(J):
        for i in range(I):
            a, b, c, d = orc.vadv_system(hp, f64["wcon"], hp, f64["utens"], f64["utens_stage"], i, j, K=K)
            out[:, j, i] = 0.15 * (orc.thomas(a, b, c, d, extended=True) - hp[:, j + 1, i + 1])
    return out


def check_plan_vs_oracle(G, orc, shapes, dtype, prec, tol):
    """Every member's h and output against the oracle composition.  Binary64 outputs
    whose oracle error exceeds `tol` are judged against the extended-precision solve of
    the same system instead: where the binary64 oracle is itself more than `tol` from it
    (long, ill-conditioned columns), no other binary64 rounding order can meet `tol`
    against the oracle, and the GPU must then be within twice the oracle's own distance
    to the extended-precision solution."""
    mems = [G.member_storages(member_draws(I, J, K, q, dtype), I, J, K) for q, (I, J, K) in enumerate(shapes)]
    plan = G.BatchPlan(mems, prec=prec)
    plan.run()
    G.device_status()
    assert plan.info()["points"] == sum(I * J * K for I, J, K in shapes)
    worst_h = worst_o = 0.0
    for q, m in enumerate(mems):
        I, J, K = m["domain"]
        f = member_draws(I, J, K, q, dtype)
        rh, ro = oracle_member(orc, f)
        eh = rel_err(m["h"].numpy(), rh)
        got = region(m["out"].numpy(), (1, 1, 0), (I, J, K))
        so = s7_stats(got, ro, tol)
        print(f"member {q} {I}x{J}x{K}: h {eh:.2e}, out {so}")
        assert eh <= tol, (q, I, J, K, eh)
        if so["max_norm"] > tol and dtype == np.float64:
            ext = extended_member(orc, f, rh)
            e_oracle, e_gpu = rel_err(ro, ext), rel_err(got, ext)
            print(f"member {q}: binary64 oracle {e_oracle:.2e} and GPU {e_gpu:.2e} from the extended-precision solve")
            assert e_oracle > tol, (q, e_oracle)  # otherwise the GPU should have met tol against the oracle
            assert e_gpu <= 2 * e_oracle, (q, e_gpu, e_oracle)
        else:
            assert so["max_norm"] <= tol, (q, I, J, K, so)
        worst_h, worst_o = max(worst_h, eh), max(worst_o, so["max_norm"])
    print(f"{len(shapes)} members, {np.dtype(dtype).name} {prec}: worst h {worst_h:.3e}, worst out {worst_o:.3e}")
    plan.close()


def test_batch_full_ensemble_fp32_vs_oracle(G, orc):
    """All 48 members of the seed-0 ensemble (I = J in {48 .. 384}, K in {40, 60, 80,
    137}), FP32 storage with double-float columns, one plan: every member's h and output
    against the oracle composition (the oracle's own h fed to its vadv) on the
    FP32-rounded inputs, 1e-5.  The GPU stores h in FP32 between the two kernels; that
    rounding alone moves the oracle composition by at most 1.4e-8 on this ensemble."""
    from paper_2311_08322_b300 import inputs
    check_plan_vs_oracle(G, orc, inputs.ensemble_shapes(48, 0), np.float32, "df", 1e-5)


def test_batch_fp64_extremes_vs_oracle(G, orc):
    """FP64 storage and binary64 columns over the ensemble's extreme member shapes (the
    smallest, 48x48x40, and the largest, 384x384x137) and two between, against the
    oracle composition at 1e-12.  On the 384x384x137 member (seed 2) the binary64 oracle
    is itself 7.5e-12 from the extended-precision solve (worst column 4.4e-11): that
    member is judged against the extended-precision solve (see check_plan_vs_oracle)."""
    shapes = [(48, 48, 40), (384, 384, 137), (256, 256, 80), (96, 96, 60)]
    check_plan_vs_oracle(G, orc, shapes, np.float64, "native", 1e-12)


@pytest.mark.parametrize("cfg", [{"hdiff_tile": 1}, {"hdiff_levels": 3}, {"hdiff_levels": 0}, {"vadv_warps": 1},
                                 {"vadv_warps": 4, "ctas_per_sm": 1}])
def test_batch_configs_agree(G, cfg):
    """Tiles, K-blocking, block width and persistent grid size change only the schedule."""
    mems = ensemble(G, 5, np.float32, shapes=SHAPES[:5])
    base = G.BatchPlan([m for m, _ in mems], prec="df")
    base.run()
    G.device_status()
    ref = [(m["h"].numpy(), m["out"].numpy()) for m, _ in mems]
    other = G.BatchPlan([m for m, _ in mems], prec="df", config=cfg)
    for m, _ in mems:
        m["h"].data.fill_(np.nan)
        m["out"].data.fill_(np.nan)
    other.run()
    G.device_status()
    for (m, _), (h0, o0) in zip(mems, ref):
        I, J, K = m["domain"]
        assert np.array_equal(m["h"].numpy(), h0)
        assert np.array_equal(region(m["out"].numpy(), (1, 1, 0), (I, J, K)), region(o0, (1, 1, 0), (I, J, K)))


def test_batch_validation(G):
    mems = ensemble(G, 2, np.float32, shapes=[(48, 48, 40), (48, 48, 40)])
    ms = [m for m, _ in mems]
    bad = [dict(ms[0]), dict(ms[1])]
    bad[1]["h"] = ms[0]["in"]  # member 1 would overwrite member 0's input
    with pytest.raises(G.GtbError) as e:
        G.BatchPlan(bad, prec="df")
    assert e.value.code == -5
    big = ensemble(G, 1, np.float32, shapes=[(8, 8, 449)])
    with pytest.raises(G.GtbError) as e:
        G.BatchPlan([big[0][0]], prec="df")
    assert e.value.code == -8


def test_autotune_cache(G, tmp_path):
    from paper_2311_08322_b300 import autotune
    mems = [m for m, _ in ensemble(G, 4, np.float32, shapes=SHAPES[:4])]
    path = str(tmp_path / "tune.json")
    cfg, log = autotune.tune(mems, prec="df", cache_path=path, reps=2)
    assert not log["cached"] and set(cfg) == set(G.DEFAULT_BATCH_CONFIG)
    cfg2, log2 = autotune.tune(mems, prec="df", cache_path=path, reps=2)
    assert log2["cached"] and cfg2 == cfg
