"""GPU parity of the differentiation form: gtb_hdiff_adj, gtb_vadv_adj and the
periodic halo pair against the oracle adjoints, and the 10-step chained
torch.autograd gradient against (a) the oracle-side reference gradient (oracle
forward + oracle adjoints + numpy's periodic padding) and (b) central finite
differences on random directions."""
import numpy as np
import pytest

from helpers import region, rel_err

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


def rnd(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, shape)


# ------------------------------------------------------------------ hdiff_adj
@pytest.mark.parametrize("I,J,K,dtype", [(256, 256, 80, np.float64), (67, 19, 5, np.float64), (1, 1, 1, np.float64),
                                         (130, 40, 3, np.float32), (64, 16, 2, np.float32)])
def test_hdiff_adj(G, orc, I, J, K, dtype):
    o = (2, 2, 0)
    shp = (K, J + 4, I + 4)
    inp, coeff, ob = rnd(shp, 1), rnd(shp, 2, 0, 0.025), rnd(shp, 3)
    inp, coeff, ob = (x.astype(dtype) for x in (inp, coeff, ob))
    cb0 = rnd(shp, 4).astype(dtype)
    s_in, s_cf, s_ob = (G.storage_from(x, o) for x in (inp, coeff, ob))
    s_ib = G.storage_from(np.full(shp, np.nan, dtype), o)
    s_cb = G.storage_from(cb0, o)
    G.hdiff_adj(s_in, s_cf, s_ob, s_ib, s_cb, accumulate=True)
    G.device_status()
    ref_cb = cb0.astype(np.float64).copy()
    ref_ib = orc.hdiff_adj(inp.astype(np.float64), coeff.astype(np.float64), ob.astype(np.float64), coeff_bar=ref_cb)
    tol = F64_TOL if dtype == np.float64 else F32_TOL
    ring = (slice(None), slice(0, J + 4), slice(0, I + 4))
    assert rel_err(s_ib.numpy()[ring], ref_ib[ring]) <= tol
    assert rel_err(region(s_cb.numpy(), o, (I, J, K)), region(ref_cb, o, (I, J, K))) <= tol


def test_hdiff_adj_overwrite_and_closed_form(G, orc):
    """Checkerboard: every flux limited, so in_bar = out_bar (0 on the ring) and coeff_bar = 0."""
    I, J, K = 40, 24, 2
    _, y, x = np.meshgrid(np.arange(K), np.arange(J + 4), np.arange(I + 4), indexing="ij")
    inp = np.where((x + y) % 2 == 0, 1.0, -1.0)
    ob = rnd(inp.shape, 5)
    o = (2, 2, 0)
    s_ib = G.storage_from(np.full(inp.shape, 7.0), o)
    s_cb = G.storage_from(np.full(inp.shape, 7.0), o)
    G.hdiff_adj(G.storage_from(inp, o), G.storage_from(rnd(inp.shape, 6, 0, 0.025), o), G.storage_from(ob, o), s_ib, s_cb)
    expect = np.zeros_like(ob)
    expect[:, 2:-2, 2:-2] = ob[:, 2:-2, 2:-2]
    assert np.array_equal(s_ib.numpy(), expect)
    assert np.all(region(s_cb.numpy(), o, (I, J, K)) == 0.0)


# ------------------------------------------------------------------ vadv_adj
@pytest.mark.parametrize("I,J,K,dtype,prec,workspace", [
    (256, 256, 80, np.float64, "native", "auto"), (70, 9, 137, np.float64, "native", None),
    (33, 7, 1, np.float64, "native", "auto"), (31, 5, 2, np.float64, "native", None),
    (200, 64, 80, np.float32, "df", "auto"), (45, 7, 30, np.float32, "f64", None)])
def test_vadv_adj(G, orc, I, J, K, dtype, prec, workspace):
    o = (1, 1, 0)
    shp = (K, J + 2, I + 2)
    wamp = 0.5 if dtype == np.float64 else 0.3
    wcon, yb = rnd(shp, 7, -wamp, wamp).astype(dtype), rnd(shp, 8).astype(dtype)
    outs = [G.storage_from(np.full(shp, np.nan, dtype), o) for _ in range(4)]
    G.vadv_adj(G.storage_from(wcon, o), G.storage_from(yb, o), *outs, prec=prec, workspace=workspace)
    G.device_status()
    refs = orc.vadv_adj(wcon.astype(np.float64), yb.astype(np.float64))
    tol = F64_TOL if dtype == np.float64 else F32_TOL
    for name, s, r in zip(("u_stage_bar", "u_pos_bar", "utens_bar", "utens_stage_bar"), outs, refs):
        assert rel_err(region(s.numpy(), o, (I, J, K)), region(r, o, (I, J, K))) <= tol, name


def test_vadv_adj_merged_and_accumulated(G, orc):
    """One storage as u_stage_bar and u_pos_bar receives their sum; GTB_ADJ_ACCUMULATE adds."""
    I, J, K = 96, 20, 40
    o = (1, 1, 0)
    shp = (K, J + 2, I + 2)
    wcon, yb, base = rnd(shp, 9, -0.5, 0.5), rnd(shp, 10), rnd(shp, 11)
    s = G.storage_from(base, o)
    G.vadv_adj(G.storage_from(wcon, o), G.storage_from(yb, o), s, s, accumulate=True)
    G.device_status()
    us, up, _, _ = orc.vadv_adj(wcon, yb)
    assert rel_err(region(s.numpy(), o, (I, J, K)), region(base + us + up, o, (I, J, K))) <= F64_TOL


# ------------------------------------------------------------------ halos
def test_halo_periodic_pair(G):
    I, J, K = 37, 21, 3
    inner = rnd((K, J, I), 12)
    s = G.storage_from(np.pad(inner, ((0, 0), (2, 2), (2, 2))), (2, 2, 0))
    G.halo_periodic(s, 2, 2)
    G.device_status()
    assert np.array_equal(s.numpy(), np.pad(inner, ((0, 0), (2, 2), (2, 2)), mode="wrap"))
    # adjoint: <P x, y> = <x, P^T y> with P the refresh
    y = rnd((K, J + 4, I + 4), 13)
    t = G.storage_from(y, (2, 2, 0))
    G.halo_periodic_adj(t, 2, 2)
    G.device_status()
    lhs = np.sum(np.pad(inner, ((0, 0), (2, 2), (2, 2)), mode="wrap") * y)
    rhs = np.sum(inner * t.numpy()[:, 2:-2, 2:-2])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ------------------------------------------------------------------ chain
def oracle_chain_grad(orc, field, coeff, wcon, utens, utens_stage, steps):
    """Loss 1/2 |final|^2 and its gradient in (field, coeff) from the oracle alone."""
    K, J, I = field.shape
    wrap2 = lambda a: np.pad(a, ((0, 0), (2, 2), (2, 2)), mode="wrap")
    pad1 = lambda a: np.pad(a, ((0, 0), (1, 1), (1, 1)))
    pad2 = lambda a: np.pad(a, ((0, 0), (2, 2), (2, 2)))
    cst = pad2(coeff)
    saved, x = [], field
    for _ in range(steps):
        st = wrap2(x)
        saved.append(st)
        h = orc.hdiff(st, cst)[:, 2:-2, 2:-2]
        x = orc.vadv(pad1(h), wcon, pad1(h), pad1(utens), pad1(utens_stage))[:, 1:-1, 1:-1]
    loss = 0.5 * np.sum(x * x)
    yb, cbar = x.copy(), np.zeros_like(coeff)
    jj, ii = np.meshgrid((np.arange(J + 4) - 2) % J, (np.arange(I + 4) - 2) % I, indexing="ij")
    for st in reversed(saved):
        us, up, _, _ = orc.vadv_adj(wcon, pad1(yb))
        hb = (us + up)[:, 1:-1, 1:-1]
        cb = np.zeros_like(cst)
        ib = orc.hdiff_adj(st, cst, pad2(hb), coeff_bar=cb)
        folded = np.zeros_like(field)
        for k in range(K):
            np.add.at(folded[k], (jj, ii), ib[k])
        yb = folded
        cbar += cb[:, 2:-2, 2:-2]
    return loss, yb, cbar


def gpu_chain(G, field, coeff, fixed, steps):
    import torch
    from paper_2311_08322_b300.autograd import chain
    f = field.clone().requires_grad_(True)
    c = coeff.clone().requires_grad_(True)
    y = chain(f, c, fixed, steps)
    loss = 0.5 * (y.double() ** 2).sum()
    loss.backward()
    return float(loss.detach()), f.grad, c.grad


def test_literal_chain_forward_vs_oracle(G, orc):
    """The 10-step chain at 256x256x80 FP64 with wcon ~ U(-0.5, 0.5) as drawn (seed 0): the
    field grows by about 1e4 per step (max |field| 3.07e4 after one step, 9.0e40 after ten).
    Every step, applied by the oracle to the GPU's own input of that step (periodic halo,
    hdiff, then vadv of h), matches the GPU's step within 1e-12 of its max-norm; over n
    steps each step's rounding adds to the last (the dominant mode carries earlier errors
    along), so the GPU chain matches the oracle's own chain within n x 1e-12."""
    import torch
    from paper_2311_08322_b300.autograd import chain, chain_inputs
    field, coeff, fixed, f = chain_inputs(256, 256, 80, seed=0, dtype=torch.float64, wcon_amp=0.5)
    fixed.save_factors = False
    wrap2 = lambda a: np.pad(a, ((0, 0), (2, 2), (2, 2)), mode="wrap")
    pad1 = lambda a: np.pad(a, ((0, 0), (1, 1), (1, 1)))
    cst = np.pad(coeff.cpu().numpy(), ((0, 0), (2, 2), (2, 2)))
    ut, uts = pad1(f["utens"][:, 1:-1, 1:-1]), pad1(f["utens_stage"][:, 1:-1, 1:-1])

    def oracle_step(x):
        h = orc.hdiff(wrap2(x), cst)[:, 2:-2, 2:-2]
        return orc.vadv(pad1(h), f["wcon"], pad1(h), ut, uts)[:, 1:-1, 1:-1]

    x, xr = field, field.cpu().numpy()
    growth = []
    with torch.no_grad():
        for step in range(1, 11):
            x_prev = x.cpu().numpy()
            x = chain(x, coeff, fixed, 1)
            got = x.cpu().numpy()
            xr = oracle_step(xr)
            assert np.all(np.isfinite(xr))
            e_step = rel_err(got, oracle_step(x_prev))
            e_chain = rel_err(got, xr)
            growth.append(float(np.abs(xr).max()))
            print(f"literal chain step {step}: max|field| {growth[-1]:.3e}, this step vs oracle {e_step:.2e}, "
                  f"chain vs oracle chain {e_chain:.2e}")
            assert e_step <= F64_TOL, (step, e_step)
            assert e_chain <= step * F64_TOL, (step, e_chain)
    assert growth[-1] > 1e40 and all(b > 1e3 * a for a, b in zip(growth, growth[1:]))


@pytest.mark.parametrize("I,J,K", [(64, 48, 40), (256, 256, 80)])
def test_chain_gradient_vs_oracle(G, orc, I, J, K):
    import torch
    from paper_2311_08322_b300.autograd import chain_inputs
    field, coeff, fixed, f = chain_inputs(I, J, K, seed=3, dtype=torch.float64)
    loss, gf, gc = gpu_chain(G, field, coeff, fixed, 10)
    rl, rf, rc = oracle_chain_grad(orc, field.cpu().numpy(), coeff.cpu().numpy(), f["wcon"],
                                   f["utens"][:, 1:-1, 1:-1], f["utens_stage"][:, 1:-1, 1:-1], 10)
    assert abs(loss - rl) <= 1e-11 * abs(rl)
    assert rel_err(gf.cpu().numpy(), rf) <= 1e-10
    assert rel_err(gc.cpu().numpy(), rc) <= 1e-10


def test_chain_gradient_fp32_vs_oracle(G, orc):
    import torch
    from paper_2311_08322_b300.autograd import chain_inputs
    I, J, K = 128, 96, 80
    field, coeff, fixed, f = chain_inputs(I, J, K, seed=4, dtype=torch.float32)
    loss, gf, gc = gpu_chain(G, field, coeff, fixed, 10)
    f32 = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
    rl, rf, rc = oracle_chain_grad(orc, field.double().cpu().numpy(), coeff.double().cpu().numpy(), f32["wcon"],
                                   f32["utens"][:, 1:-1, 1:-1], f32["utens_stage"][:, 1:-1, 1:-1], 10)
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    assert rel_err(gf.cpu().numpy(), rf) <= 1e-4
    assert rel_err(gc.cpu().numpy(), rc) <= 1e-4


def limiter_keep_masks(x):
    """The limiter decisions hdiff takes on one chain step's input x (interior (K, J, I),
    its 2-point halo refreshed periodically): for every flux of the definition, whether it
    is kept (fx * (in[i+1] - in[i]) > 0 zeroes it; fy likewise).  Computed with torch ops
    on the device, for flagging finite-difference directions that cross a decision."""
    import torch
    xs = torch.cat([x[:, :, -2:], x, x[:, :, :2]], dim=2)
    xs = torch.cat([xs[:, -2:], xs, xs[:, :2]], dim=1)  # (K, J+4, I+4)
    c = xs[:, 1:-1, 1:-1]
    lap = 4 * c - (((xs[:, 1:-1, 2:] + xs[:, 1:-1, :-2]) + xs[:, 2:, 1:-1]) + xs[:, :-2, 1:-1])  # i, j in [-1, I]
    fx = lap[:, 1:-1, 1:] - lap[:, 1:-1, :-1]       # i in [-1, I-1], j in [0, J)
    gx = c[:, 1:-1, 1:] - c[:, 1:-1, :-1]
    fy = lap[:, 1:, 1:-1] - lap[:, :-1, 1:-1]       # i in [0, I), j in [-1, J-1]
    gy = c[:, 1:, 1:-1] - c[:, :-1, 1:-1]
    return ~(fx * gx > 0), ~(fy * gy > 0)


@pytest.mark.parametrize("I,J,K", [(64, 48, 40), (256, 256, 80)])
def test_chain_gradient_central_differences(G, I, J, K):
    """32 random unit directions in (field, coeff), h = 1e-6, 10 chained steps, FP64.  The
    loss is piecewise polynomial in the inputs (one piece per set of limiter decisions), so
    central differences are exact up to rounding unless a decision switches inside
    [-h, h]: such directions are flagged (at any step, a flux kept at one end and zeroed at
    the other, or at the centre) and set aside.  The loss difference is formed as
    sum((x+ - x-)(x+ + x-)) / 2, not as the difference of two sums of squares, whose own
    rounding (about 1e-8 at 256x256x80, where the loss is ~1e7) would swamp a step of 1e-6.
    Every unflagged direction must agree, and at least 16 of 32 must be unflagged."""
    import torch
    from paper_2311_08322_b300.autograd import chain, chain_inputs
    field, coeff, fixed, _ = chain_inputs(I, J, K, seed=5, dtype=torch.float64)
    _, gf, gc = gpu_chain(G, field, coeff, fixed, 10)
    rng = np.random.default_rng(6)
    fixed.save_factors = False  # forward-only runs below

    def run(df, dc):
        """Final field and the limiter decisions of every step."""
        masks, x = [], field + df
        with torch.no_grad():
            for _ in range(10):
                masks.append(limiter_keep_masks(x))
                x = chain(x, coeff + dc, fixed, 1)
        return x, masks

    def crosses(ma, mb):
        return any(not torch.equal(a[0], b[0]) or not torch.equal(a[1], b[1]) for a, b in zip(ma, mb))

    _, m0 = run(torch.zeros_like(field), torch.zeros_like(coeff))
    good, worst = 0, 0.0
    for d in range(32):
        vf = torch.from_numpy(rng.standard_normal(field.shape)).cuda()
        vc = torch.from_numpy(rng.standard_normal(coeff.shape)).cuda() * 1e-2
        nrm = torch.sqrt((vf ** 2).sum() + (vc ** 2).sum())
        vf, vc = vf / nrm, vc / nrm
        h = 1e-6
        xp, mp = run(h * vf, h * vc)
        xm, mm = run(-h * vf, -h * vc)
        if crosses(mp, m0) or crosses(mm, m0):
            print(f"direction {d}: a limiter decision switches within [-h, h]; set aside")
            continue
        fd = float(((xp - xm) * (xp + xm)).sum()) / (4 * h)
        exact = float((gf * vf).sum() + (gc * vc).sum())
        err = abs(fd - exact) / max(1.0, abs(exact))
        worst = max(worst, err)
        print(f"direction {d}: fd {fd:.12e} adjoint {exact:.12e} rel {err:.2e}")
        assert err <= 1e-5, (d, fd, exact)
        good += 1
    print(f"{good} of 32 directions unflagged, worst relative difference {worst:.2e}")
    assert good >= 16, good
    # Random unit directions in ~10M dimensions see directional derivatives of ~1e-3, where the
    # criterion above is effectively absolute.  Along the gradient itself, v = g / |g|, the
    # derivative is |g| (order 1 to 10 here): a relative check of the gradient's length and
    # direction at once (a wrong term of either sign changes |g| and the central difference
    # along it differently).
    gn = torch.sqrt((gf ** 2).sum() + (gc ** 2).sum())
    vf, vc = gf / gn, gc / gn
    h = 1e-6
    xp, mp = run(h * vf, h * vc)
    xm, mm = run(-h * vf, -h * vc)
    if crosses(mp, m0) or crosses(mm, m0):
        print("gradient direction: a limiter decision switches within [-h, h]; set aside")
        return
    fd = float(((xp - xm) * (xp + xm)).sum()) / (4 * h)
    rel = abs(fd - float(gn)) / float(gn)
    print(f"gradient direction: fd {fd:.12e} |g| {float(gn):.12e} rel {rel:.2e}")
    assert rel <= 1e-5, (fd, float(gn))


@pytest.mark.parametrize("dtype,prec", [(np.float64, "native"), (np.float32, "df"), (np.float32, "f64"),
                                        (np.float32, "native")])
@pytest.mark.parametrize("I,J,K", [(70, 33, 41), (33, 7, 1), (31, 5, 2)])
def test_adjoint_from_kept_factors(G, dtype, prec, I, J, K):
    """gtb_hdiff_vadv with GTB_SAVE_FACTORS returns the same output, and gtb_vadv_adj
    on the kept factors (GTB_ADJ_FACTORS) the same cotangents as the refactorising
    adjoint, bit for bit (the same pivots and c' values), merged and separate."""
    import torch
    from paper_2311_08322_b300 import inputs
    f = inputs.hdiff_vadv(I, J, K, seed=12)
    dom = (I, J, K)
    s = {n: G.storage_from(f[n].astype(dtype), (2, 2, 0) if n in ("in", "coeff") else (1, 1, 0))
         for n in ("in", "coeff", "wcon", "utens", "utens_stage", "u_pos")}
    zeros = lambda: G.storage_from(np.zeros_like(f["utens"]).astype(dtype), (1, 1, 0))
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    for merge in (True, False):
        o1, o2 = zeros(), zeros()
        F = torch.empty(G.hdiff_vadv_workspace_bytes(tdt, prec, dom, save_factors=True), dtype=torch.uint8,
                        device="cuda")
        G.hdiff_vadv(s["in"], s["coeff"], s["wcon"], s["utens"], s["utens_stage"], o1, prec=prec, domain=dom)
        G.hdiff_vadv(s["in"], s["coeff"], s["wcon"], s["utens"], s["utens_stage"], o2, prec=prec, domain=dom,
                     workspace=F, save_factors=True)
        a1, b1, c1, a2, b2, c2 = (zeros() for _ in range(6))
        if merge:
            G.vadv_adj(s["wcon"], s["u_pos"], a1, a1, c1, prec=prec, domain=dom)
            G.vadv_adj(s["wcon"], s["u_pos"], a2, a2, c2, prec=prec, domain=dom, workspace=F, factors=True)
        else:
            G.vadv_adj(s["wcon"], s["u_pos"], a1, b1, c1, prec=prec, domain=dom)
            G.vadv_adj(s["wcon"], s["u_pos"], a2, b2, c2, prec=prec, domain=dom, workspace=F, factors=True)
        G.device_status()
        assert np.array_equal(o1.numpy(), o2.numpy())
        for x, y in ((a1, a2), (b1, b2), (c1, c2)):
            assert np.array_equal(x.numpy(), y.numpy()), (merge, prec)


def test_chain_gradient_with_and_without_factors(G):
    """The differentiable chain keeps each step's factors by default; without them the
    backward refactorises: the same gradients, bit for bit."""
    import torch
    from paper_2311_08322_b300.autograd import chain_inputs
    field, coeff, fixed, _ = chain_inputs(64, 40, 30, seed=4, dtype=torch.float64)
    l1, gf1, gc1 = gpu_chain(G, field, coeff, fixed, 4)
    fixed.save_factors = False
    l2, gf2, gc2 = gpu_chain(G, field, coeff, fixed, 4)
    assert l1 == l2
    assert torch.equal(gf1, gf2) and torch.equal(gc1, gc2)


@pytest.mark.parametrize("beta_v,literal,merge", [(0.3, False, False), (-0.2, True, False), (0.3, False, True),
                                                  (0.0, True, False), (0.0, False, True)])
def test_vadv_adj_weights(G, orc, beta_v, literal, merge):
    """Both bodies of the backward sweep: beta_v = 0 (u_stage_bar = dtr (z - y_bar), no
    wcon read) and general weights (the E^T z stencil), separate and merged cotangents,
    against the oracle's adjoint.  A literal face velocity is wcon(i) itself, not an average
    of two: |wcon| <= 0.25 keeps its columns as well conditioned as the averaged draws (at
    0.5 some diagonals turn negative and the binary64 oracle itself is 8e-12 from a
    long-double solve, so no other rounding order can meet 1e-12 against it)."""
    I, J, K = 70, 11, 37
    o = (1, 1, 0)
    shp = (K, J + 2, I + 2)
    amp = 0.25 if literal else 0.5
    wcon, yb = rnd(shp, 21, -amp, amp), rnd(shp, 22)
    us, up, ut, uts = orc.vadv_adj(wcon, yb, beta_v=beta_v, wmode=1 if literal else 0)
    kw = dict(beta_v=beta_v, literal=literal)
    if merge:
        s = G.storage_from(np.full(shp, np.nan), o)
        G.vadv_adj(G.storage_from(wcon, o), G.storage_from(yb, o), s, s, **kw)
        G.device_status()
        assert rel_err(region(s.numpy(), o, (I, J, K)), region(us + up, o, (I, J, K))) <= F64_TOL
        return
    outs = [G.storage_from(np.full(shp, np.nan), o) for _ in range(4)]
    G.vadv_adj(G.storage_from(wcon, o), G.storage_from(yb, o), *outs, **kw)
    G.device_status()
    for name, st, r in zip(("u_stage_bar", "u_pos_bar", "utens_bar", "utens_stage_bar"), outs, (us, up, ut, uts)):
        assert rel_err(region(st.numpy(), o, (I, J, K)), region(r, o, (I, J, K))) <= F64_TOL, name
