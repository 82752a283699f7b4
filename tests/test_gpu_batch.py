"""GPU tests of the batched form: an ensemble of uneven domains run by two
persistent kernels replayed from a CUDA graph (gtb_batch_plan / gtb_batch_run).
Each member computes h = hdiff(in, coeff), out = vadv(h, wcon, h, utens,
utens_stage).  Results must equal the single-domain entry points bit for bit
(same per-point arithmetic) and the oracle within the bounds."""
import numpy as np
import pytest

from helpers import region, rel_err

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


def test_batch_vs_oracle(G, orc):
    shapes = [(48, 48, 40), (96, 96, 137), (128, 128, 60)]
    mems = ensemble(G, 3, np.float32, shapes=shapes)
    plan = G.BatchPlan([m for m, _ in mems], prec="df")
    plan.run()
    G.device_status()
    for m, f in mems:
        I, J, K = m["domain"]
        h = m["h"].numpy()
        ref_h = orc.hdiff(f["in"].astype(np.float64), f["coeff"].astype(np.float64))[:, 2:-2, 2:-2]
        assert rel_err(h, ref_h) <= 1e-5
        hp = np.pad(h.astype(np.float64), ((0, 0), (1, 1), (1, 1)))
        ref = orc.vadv(hp, f["wcon"].astype(np.float64), hp, f["utens"].astype(np.float64),
                       f["utens_stage"].astype(np.float64))
        assert rel_err(region(m["out"].numpy(), (1, 1, 0), (I, J, K)), region(ref, (1, 1, 0), (I, J, K))) <= 1e-5


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
