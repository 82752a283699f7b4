"""Pins of the hdiff oracle against closed forms and exact symmetries.

hdiff is the paper's horizontal-diffusion benchmark (Sec. 3.1), a PARALLEL
computation with if-else bodies (Sec. 2.2): Laplacian, flux-limited fluxes,
update.  None of these tests calls the oracle twice to check it against
itself with retyped formulas; each expected value is a closed form derived
by hand (derivations in the docstrings) or an exact symmetry.
"""
import numpy as np
import pytest

H = 2  # hdiff halo


def grid(I, J, K):
    """Storage coordinates x (= i) and y (= j), broadcast to (K, J+4, I+4)."""
    k, y, x = np.meshgrid(np.arange(K), np.arange(J + 2 * H), np.arange(I + 2 * H), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64)


def dyadic_coeff(rng, shape):
    """coeff in [0, 0.025) on a 2^-10 lattice, so products with small integers are exact."""
    return rng.integers(0, 26, size=shape).astype(np.float64) / 1024.0


def inner(a):
    return a[:, H:-H, H:-H]


@pytest.mark.parametrize("c", [0.0, 1.0, -0.7316, 3.5e5])
def test_constant_field_unchanged(orc, c):
    """W1: lap = 4c - 4c = 0, so every flux vanishes and out = in exactly."""
    rng = np.random.default_rng(1)
    inp = np.full((5, 12, 14), c)
    coeff = rng.uniform(0, 0.025, inp.shape)
    out = orc.hdiff(inp, coeff)
    assert np.array_equal(inner(out), inner(inp))


def test_quadratic_field_unchanged(orc):
    """W2: in = a x^2 + b y^2 + g xy + d x has lap = -2(a+b) everywhere, so fx = fy = 0."""
    x, y = grid(11, 9, 3)
    inp = 0.25 * x * x - 0.125 * y * y + 0.5 * x * y + 0.75 * x
    coeff = dyadic_coeff(np.random.default_rng(2), inp.shape)
    out = orc.hdiff(inp, coeff)
    assert np.array_equal(inner(out), inner(inp))


@pytest.mark.parametrize("axis", ["i", "j"])
def test_quartic_field(orc, axis):
    """W3: in = x^4 gives lap = -(12x^2+2), fx = -12(2x+1); fx*(in[x+1]-in[x]) < 0 for every
    integer x, so no flux is limited, and fx[x]-fx[x-1] = -24: out = in + 24 coeff exactly.
    The same holds along j for in = y^4 (pins the fy branch)."""
    I, J, K = 13, 10, 4
    x, y = grid(I, J, K)
    t = (x - 7.0) if axis == "i" else (y - 5.0)
    inp = t ** 4
    coeff = dyadic_coeff(np.random.default_rng(3), inp.shape)
    out = orc.hdiff(inp, coeff)
    assert np.array_equal(inner(out), inner(inp + 24.0 * coeff))


def test_checkerboard_fully_limited(orc):
    """W4: in = s = (-1)^(i+j): lap = 8s, fx = -16s, in[i+1]-in[i] = -2s, product 32 > 0:
    every flux is limited, out = in.  (Unlimited it would be in + 64 coeff in.)"""
    x, y = grid(10, 12, 3)
    inp = np.where((x + y) % 2 == 0, 1.0, -1.0)
    coeff = np.random.default_rng(4).uniform(0, 0.025, inp.shape)
    out = orc.hdiff(inp, coeff)
    assert np.array_equal(inner(out), inner(inp))


@pytest.mark.parametrize("axis", ["i", "j"])
def test_unit_step_strict_limiter(orc, axis):
    """W5: unit step at storage index s0.  Hand derivation (tests/golden/hdiff_unit_step.txt):
    out - in = +c, -c, +c, -c at s0-2, s0-1, s0, s0+1 and 0 elsewhere.  A limiter that also
    fired on a zero product (>= 0) would give 0 everywhere; one with the wrong sign gives
    (+c, -3c, +3c, -c)."""
    I, J, K = 12, 11, 2
    x, y = grid(I, J, K)
    s0 = 8
    t = x if axis == "i" else y
    inp = (t >= s0).astype(np.float64)
    coeff = dyadic_coeff(np.random.default_rng(5), inp.shape) + 1.0 / 1024
    out = orc.hdiff(inp, coeff)
    golden = np.loadtxt(__file__.replace("test_oracle_hdiff.py", "golden/hdiff_unit_step.txt"))
    pattern = np.zeros_like(inp)
    for off, sgn in golden:
        pattern = np.where(t == s0 + off, sgn, pattern)
    assert np.array_equal(inner(out - inp), inner(pattern * coeff))


def test_reflection_symmetry_exact(orc):
    """Mirroring i (or j) maps every forward difference to minus the mirrored one, so the
    limiter products are unchanged and hdiff commutes with the mirror bit for bit."""
    rng = np.random.default_rng(6)
    inp = rng.uniform(-1, 1, (6, 17, 15))
    coeff = rng.uniform(0, 0.025, inp.shape)
    out = orc.hdiff(inp, coeff)
    for ax in (1, 2):
        outm = orc.hdiff(np.ascontiguousarray(np.flip(inp, ax)), np.ascontiguousarray(np.flip(coeff, ax)))
        assert np.array_equal(inner(outm), inner(np.flip(out, ax)))


def test_transpose_symmetry(orc):
    """Swapping i and j swaps fx and fy; only the summation order of lap changes."""
    rng = np.random.default_rng(7)
    inp = rng.uniform(-1, 1, (4, 16, 16))
    coeff = rng.uniform(0, 0.025, inp.shape)
    out = orc.hdiff(inp, coeff)
    outt = orc.hdiff(np.ascontiguousarray(inp.transpose(0, 2, 1)), np.ascontiguousarray(coeff.transpose(0, 2, 1)))
    np.testing.assert_allclose(inner(outt), inner(out.transpose(0, 2, 1)), rtol=0, atol=1e-15)


def test_positive_power_of_two_scaling(orc):
    """hdiff is positively homogeneous: scaling in by 2^m scales every flux, every limiter
    product by 2^(2m) > 0, and the update by 2^m, all exactly."""
    rng = np.random.default_rng(8)
    inp = rng.uniform(-1, 1, (3, 14, 18))
    coeff = rng.uniform(0, 0.025, inp.shape)
    out = orc.hdiff(inp, coeff)
    for s in (2.0 ** -7, 2.0 ** 9, -(2.0 ** 3)):
        assert np.array_equal(inner(orc.hdiff(inp * s, coeff)), inner(out * s))


def test_origin_and_domain_plumbing(orc):
    """A sub-domain with its own origins equals the matching slice of a full call."""
    rng = np.random.default_rng(9)
    inp = rng.uniform(-1, 1, (5, 20, 24))
    coeff = rng.uniform(0, 0.025, inp.shape)
    full = orc.hdiff(inp, coeff)
    out = np.zeros((3, 7, 9))
    orc.hdiff(inp, coeff, out, origin_in=(5, 4, 1), origin_coeff=(5, 4, 1), origin_out=(0, 0, 0),
              domain=(9, 7, 3))
    assert np.array_equal(out, full[1:4, 4:11, 5:14])


def test_extent_check(orc):
    inp = np.zeros((2, 8, 8))
    with pytest.raises(ValueError):
        orc.hdiff(inp, inp.copy(), origin_in=(1, 2, 0), domain=(4, 4, 2))
