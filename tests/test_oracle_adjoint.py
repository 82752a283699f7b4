"""Pins of the adjoint oracles (reverse-mode hdiff and vadv) against the forward
oracle: dot-product identities <J v, w> = <v, J^T w>, Jacobians materialised
column by column and transposed, and closed forms.  vadv is linear in
(u_stage, u_pos, utens, utens_stage) for fixed wcon; hdiff is linear on each
piece of the limiter (masks frozen at the forward input) and exactly linear in
coeff."""
import numpy as np
import pytest

DTR = 0.15
VN = ("u_stage", "u_pos", "utens", "utens_stage")


def rnd(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, shape)


def vadv_lin(orc, wcon, v):
    return orc.vadv(v["u_stage"], wcon, v["u_pos"], v["utens"], v["utens_stage"])


@pytest.mark.parametrize("wamp,K,tol", [(0.15, 30, 1e-13), (0.5, 80, 1e-9)])
def test_vadv_dot_product(orc, wamp, K, tol):
    I, J = 9, 7
    shp = (K, J + 2, I + 2)
    wcon = rnd(shp, 1, -wamp, wamp)
    v = {n: rnd(shp, 10 + q) for q, n in enumerate(VN)}
    w = rnd(shp, 20)
    w[:, 0, :] = w[:, -1, :] = 0.0
    w[:, :, 0] = w[:, :, -1] = 0.0       # only the domain carries cotangents
    Jv = vadv_lin(orc, wcon, v)
    us_b, up_b, ut_b, uts_b = orc.vadv_adj(wcon, w)
    lhs = np.sum(Jv[:, 1:-1, 1:-1] * w[:, 1:-1, 1:-1])
    rhs = sum(np.sum(b[:, 1:-1, 1:-1] * v[n][:, 1:-1, 1:-1]) for b, n in zip((us_b, up_b, ut_b, uts_b), VN))
    assert abs(lhs - rhs) <= tol * (abs(lhs) + 1.0)
    assert np.array_equal(ut_b, uts_b)


@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_vadv_materialised_jacobian(orc, K):
    """Build J column by column from the forward oracle (unit inputs), transpose it,
    and compare J^T w with the adjoint oracle for every input field."""
    I, J = 2, 1
    shp = (K, J + 2, I + 2)
    wcon = rnd(shp, 30 + K, -0.4, 0.4)
    w = np.zeros(shp)
    w[:, 1:-1, 1:-1] = rnd((K, J, I), 40 + K)
    bars = dict(zip(VN, orc.vadv_adj(wcon, w)))
    dom = [(k, j + 1, i + 1) for k in range(K) for j in range(J) for i in range(I)]
    for n in VN:
        Jm = np.zeros((len(dom), len(dom)))
        for c, idx in enumerate(dom):
            v = {m: np.zeros(shp) for m in VN}
            v[n][idx] = 1.0
            y = vadv_lin(orc, wcon, v)
            Jm[:, c] = [y[p] for p in dom]
        expect = Jm.T @ np.array([w[p] for p in dom])
        got = np.array([bars[n][p] for p in dom])
        np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-13)


def test_hdiff_checkerboard_adjoint_is_identity(orc):
    """Every flux of (-1)^(i+j) is limited, so out = in locally and in_bar = out_bar on
    the domain, 0 on the ring; D = 0 so coeff_bar = 0."""
    K, J, I = 2, 10, 12
    _, y, x = np.meshgrid(np.arange(K), np.arange(J + 4), np.arange(I + 4), indexing="ij")
    inp = np.where((x + y) % 2 == 0, 1.0, -1.0)
    coeff = rnd(inp.shape, 2, 0, 0.025)
    ob = rnd(inp.shape, 3)
    cb = np.zeros_like(coeff)
    ib = orc.hdiff_adj(inp, coeff, ob, coeff_bar=cb)
    expect = np.zeros_like(ob)
    expect[:, 2:-2, 2:-2] = ob[:, 2:-2, 2:-2]
    assert np.array_equal(ib, expect)
    assert np.all(cb == 0.0)


def hdiff_inner(orc, inp, coeff):
    return orc.hdiff(inp, coeff)[:, 2:-2, 2:-2]


def test_hdiff_dot_product_unlimited_field(orc):
    """in = x^4 + y^4 (no flux limited, margins >= 12 per flux): small perturbations keep
    every mask, so finite differences with a power-of-two step give J v exactly up to
    rounding; <J v, w> = <v, J^T w>."""
    K, J, I = 3, 11, 13
    _, y, x = np.meshgrid(np.arange(K), np.arange(J + 4), np.arange(I + 4), indexing="ij")
    inp = (x - 7.0) ** 4 + (y - 6.0) ** 4
    coeff = rnd(inp.shape, 4, 0, 0.025)
    v = rnd(inp.shape, 5)
    w = np.zeros_like(inp)
    w[:, 2:-2, 2:-2] = rnd((K, J, I), 6)
    eps = 2.0 ** -12
    Jv = (hdiff_inner(orc, inp + eps * v, coeff) - hdiff_inner(orc, inp - eps * v, coeff)) / (2 * eps)
    ib = orc.hdiff_adj(inp, coeff, w)
    lhs = np.sum(Jv * w[:, 2:-2, 2:-2])
    rhs = np.sum(ib * v)
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_hdiff_materialised_jacobian_random(orc):
    """Tiny random field: central-difference Jacobian column by column (a column whose
    step crosses a limiter switch is detected by comparing steps h and h/2 and must
    not occur), transposed, against the adjoint oracle on the whole 2-ring."""
    K, J, I = 1, 3, 4
    shp = (K, J + 4, I + 4)
    inp = rnd(shp, 7)
    coeff = rnd(shp, 8, 0, 0.025)
    w = np.zeros(shp)
    w[:, 2:-2, 2:-2] = rnd((K, J, I), 9)
    ib = orc.hdiff_adj(inp, coeff, w)
    h = 1e-7
    for idx in np.ndindex(shp):
        e = np.zeros(shp)
        e[idx] = 1.0
        d1 = (hdiff_inner(orc, inp + h * e, coeff) - hdiff_inner(orc, inp - h * e, coeff)) / (2 * h)
        d2 = (hdiff_inner(orc, inp + 0.5 * h * e, coeff) - hdiff_inner(orc, inp - 0.5 * h * e, coeff)) / h
        assert np.max(np.abs(d1 - d2)) < 1e-6, f"limiter switch within the step at {idx}"
        assert abs(np.sum(d1 * w[:, 2:-2, 2:-2]) - ib[idx]) < 1e-7, idx


def test_hdiff_coeff_bar_exactly_linear(orc):
    """out is linear in coeff (the masks depend on in only): out(coeff + v) - out(coeff)
    = -D v exactly, so <that, w> = <v, coeff_bar(w)>."""
    K, J, I = 2, 9, 8
    shp = (K, J + 4, I + 4)
    inp = rnd(shp, 11)
    coeff = rnd(shp, 12, 0, 0.025)
    v = rnd(shp, 13) / 64
    w = np.zeros(shp)
    w[:, 2:-2, 2:-2] = rnd((K, J, I), 14)
    cb = np.zeros(shp)
    orc.hdiff_adj(inp, coeff, w, coeff_bar=cb)
    dv = hdiff_inner(orc, inp, coeff + v) - hdiff_inner(orc, inp, coeff)
    lhs = np.sum(dv * w[:, 2:-2, 2:-2])
    rhs = np.sum(cb * v)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-3)


@pytest.mark.parametrize("wmode", [0, 1])
def test_vadv_adjoint_stage_identity(orc, wmode):
    """With beta_v = 0 the explicit operator is E = dtr I - A, and the adjoint solve
    A^T z = dtr y_bar then gives u_stage_bar = E^T z = dtr (z - y_bar) = u_pos_bar, with
    z = utens_bar: a closed form the oracle's stencil form of E^T z must reproduce (a
    dropped or mis-signed weight breaks it), while beta_v != 0 must not."""
    I, J, K = 11, 6, 24
    shp = (K, J + 2, I + 2)
    amp = 0.25 if wmode else 0.5
    wcon, yb = rnd(shp, 31, -amp, amp), rnd(shp, 32)
    us_b, up_b, ut_b, _ = orc.vadv_adj(wcon, yb, wmode=wmode)
    d = (slice(None), slice(1, -1), slice(1, -1))
    closed = DTR * (ut_b[d] - yb[d])
    scale = np.max(np.abs(closed))
    assert np.max(np.abs(us_b[d] - closed)) <= 1e-13 * scale
    assert np.max(np.abs(up_b[d] - closed)) <= 1e-13 * scale
    us_g, _, ut_g, _ = orc.vadv_adj(wcon, yb, wmode=wmode, beta_v=0.3)
    assert np.max(np.abs(us_g[d] - DTR * (ut_g[d] - yb[d]))) > 1e-6 * scale
