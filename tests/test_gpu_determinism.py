"""Race detection by repetition (compute-sanitizer is not available on this machine):
every entry point runs twice on the same inputs, with its outputs and its
workspace filled beforehand with different garbage (NaN, then huge values), and
must give the same results bit for bit on everything it writes, all finite.  A
race in a shared-memory ring or between the sweeps of a column, or a read of a
workspace slot before it is written, shows up as a difference or as garbage
leaking into the result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

VN = ("u_stage", "wcon", "u_pos", "utens", "utens_stage")


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2311_08322_b300 import build, gtb
    assert torch.cuda.is_available()
    build.build()
    return gtb


def fields(G, I, J, K, seed, dtype=np.float64):
    from paper_2311_08322_b300 import inputs
    f = inputs.hdiff_vadv(I, J, K, seed=seed)
    s = {n: G.storage_from(f[n].astype(dtype), (2, 2, 0) if n in ("in", "coeff") else (1, 1, 0))
         for n in ("in", "coeff", *VN)}
    return f, s


def region(a, origin, dom):
    (oi, oj, ok), (I, J, K) = origin, dom
    return a[ok:ok + K, oj:oj + J, oi:oi + I]


def twice(G, run, outs, ws=None):
    """outs: (storage, origin, domain) of each region the call writes.  run() twice,
    the outputs and the workspace filled first with NaN bit patterns, then with huge
    finite ones; the written regions must agree bit for bit and be finite."""
    import torch
    res = []
    for fill, byte in ((float("nan"), 0xFF), (1e300, 0x7F)):
        for st, _, _ in outs:
            st.data.fill_(fill if st.data.dtype == torch.float64 or fill != fill else 3e38)
        if ws is not None:
            ws.fill_(byte)
        run()
        G.device_status()
        res.append([region(st.numpy(), o, d) for st, o, d in outs])
    for a, b in zip(*res):
        assert np.array_equal(a, b)
        assert np.isfinite(a).all()
    return res[0]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_step_fused_and_vadv(G, dtype):
    import torch
    I, J, K = 97, 35, 41
    dom = (I, J, K)
    f, s = fields(G, I, J, K, 1, dtype)
    ho = G.storage_from(np.zeros_like(f["coeff"]).astype(dtype), (2, 2, 0))
    vo = G.storage_from(np.zeros_like(f["utens"]).astype(dtype), (1, 1, 0))
    prec = "native" if dtype == np.float64 else "df"
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    ws = torch.empty(G.hdiff_vadv_workspace_bytes(tdt, prec, dom, save_factors=True), dtype=torch.uint8,
                     device="cuda")
    twice(G, lambda: G.step(s["in"], s["coeff"], ho, *[s[n] for n in VN], vo, prec=prec, domain=dom,
                            workspace=ws), [(ho, (2, 2, 0), dom), (vo, (1, 1, 0), dom)], ws)
    twice(G, lambda: G.hdiff_vadv(s["in"], s["coeff"], s["wcon"], s["utens"], s["utens_stage"], vo, prec=prec,
                                  domain=dom, workspace=ws, save_factors=True), [(vo, (1, 1, 0), dom)], ws)
    twice(G, lambda: G.vadv(*[s[n] for n in VN], vo, prec=prec, domain=dom, workspace=ws),
          [(vo, (1, 1, 0), dom)], ws)
    twice(G, lambda: G.vadv(*[s[n] for n in VN], vo, prec=prec, domain=dom, workspace=None),
          [(vo, (1, 1, 0), dom)])


def test_adjoints(G):
    import torch
    I, J, K = 97, 35, 41
    dom = (I, J, K)
    f, s = fields(G, I, J, K, 2)
    ib = G.storage_from(np.zeros_like(f["in"]), (2, 2, 0))
    cb = G.storage_from(np.zeros_like(f["coeff"]), (2, 2, 0))
    ob = G.storage_from(np.random.default_rng(3).uniform(-1, 1, f["coeff"].shape), (2, 2, 0))
    twice(G, lambda: G.hdiff_adj(s["in"], s["coeff"], ob, ib, cb, domain=dom),
          [(ib, (0, 0, 0), (I + 4, J + 4, K)), (cb, (2, 2, 0), dom)])
    hb = G.storage_from(np.zeros_like(f["utens"]), (1, 1, 0))
    ut = G.storage_from(np.zeros_like(f["utens"]), (1, 1, 0))
    ws = torch.empty(2 * G.vadv_workspace_bytes(torch.float64, "native", dom), dtype=torch.uint8, device="cuda")
    outs = [(hb, (1, 1, 0), dom), (ut, (1, 1, 0), dom)]
    twice(G, lambda: G.vadv_adj(s["wcon"], s["u_pos"], hb, hb, ut, domain=dom, workspace=ws), outs, ws)
    twice(G, lambda: G.vadv_adj(s["wcon"], s["u_pos"], hb, hb, ut, domain=dom, workspace=None), outs)


def test_batch_plan_replay(G):
    from test_gpu_batch import ensemble
    mems = ensemble(G, 5, np.float32)
    plan = G.BatchPlan([m for m, _ in mems], prec="df")
    outs = [(m["out"], (1, 1, 0), m["domain"]) for m, _ in mems] + [(m["h"], (0, 0, 0), m["domain"]) for m, _ in mems]
    twice(G, plan.run, outs)
