"""Pins of the vadv oracle (implicit vertical advection, GT4Py paper Sec. 3.1;
FORWARD then BACKWARD computations with specialised top/bottom intervals, Sec. 2.2).

Expected values come from identities of the tridiagonal system, an exact
reversal symmetry, independent solvers (numpy's pivoted LU, exact rational
elimination, an extended-precision Thomas) and the LU backward-error bound.
"""
from fractions import Fraction

import numpy as np
import pytest

DTR = 3.0 / 20.0
EPS = np.finfo(np.float64).eps


def fields(I, J, K, seed, wamp=0.5):
    rng = np.random.default_rng(seed)
    shp = (K, J + 2, I + 2)
    f = {n: rng.uniform(-1, 1, shp) for n in ("u_stage", "u_pos", "utens", "utens_stage")}
    f["wcon"] = rng.uniform(-wamp, wamp, shp)
    return f


def run(orc, f, **kw):
    return orc.vadv(f["u_stage"], f["wcon"], f["u_pos"], f["utens"], f["utens_stage"], **kw)


def inner(a):
    return a[:, 1:-1, 1:-1]


def test_zero_velocity(orc):
    """I1: wcon = 0 makes A = dtr*Id and removes the explicit terms, so
    utens_stage_out = dtr*((dtr u_pos + utens + utens_stage)/dtr - u_pos) = utens + utens_stage."""
    f = fields(9, 7, 12, 1)
    f["wcon"][:] = 0.0
    out = run(orc, f)
    np.testing.assert_allclose(inner(out), inner(f["utens"] + f["utens_stage"]), rtol=0, atol=2e-15)


@pytest.mark.parametrize("wamp,tol", [(0.15, 1e-13), (0.5, 1e-8)])
def test_row_sum_identity(orc, wamp, tol):
    """I2: every row of A sums to dtr (b = dtr - a - c, with a_0 = c_{K-1} = 0).  With u_stage
    constant in k the explicit terms vanish, so for u_pos = P and utens + utens_stage = T
    (constant per column) the solution is x = P + T/dtr and the output is T in every level."""
    I, J, K = 8, 6, 40
    rng = np.random.default_rng(2)
    f = fields(I, J, K, 3, wamp)
    shp = f["u_pos"].shape
    P = rng.uniform(-1, 1, (1,) + shp[1:])
    T = rng.integers(-64, 64, (1,) + shp[1:]) / 64.0
    f["u_stage"] = np.broadcast_to(rng.uniform(-1, 1, (1,) + shp[1:]), shp).copy()
    f["u_pos"] = np.broadcast_to(P, shp).copy()
    f["utens"] = rng.integers(-64, 64, shp) / 128.0   # dyadic, so T - utens is exact
    f["utens_stage"] = np.broadcast_to(T, shp) - f["utens"]
    out = run(orc, f)
    np.testing.assert_allclose(inner(out), inner(np.broadcast_to(T, shp)), rtol=0, atol=tol)


@pytest.mark.parametrize("wmode", [0, 1])
def test_reversal_symmetry(orc, wmode):
    """Reversing a column (cell k -> K-1-k) maps face m to face K-m and flips the sign of the
    vertical velocity.  With u' = u[::-1] and wcon'[m] = -wcon[K-m] (m >= 1) every coefficient
    maps exactly (a'_k = c_{K-1-k}, c'_k = a_{K-1-k}), so out' = out[::-1] up to the rounding
    of the opposite elimination order.  A sign or index error in a_k/c_k breaks the symmetry."""
    I, J, K = 10, 8, 30
    f = fields(I, J, K, 4, 0.15)
    g = {n: np.ascontiguousarray(f[n][::-1]) for n in ("u_stage", "u_pos", "utens", "utens_stage")}
    w = np.zeros_like(f["wcon"])
    w[1:] = -f["wcon"][:0:-1]
    g["wcon"] = w
    out, outr = run(orc, f, wmode=wmode), run(orc, g, wmode=wmode)
    np.testing.assert_allclose(inner(outr), inner(out[::-1]), rtol=0, atol=2e-14)
    # the same transformation without the sign flip must NOT be a symmetry
    g["wcon"] = -w
    assert np.max(np.abs(inner(run(orc, g, wmode=wmode)) - inner(out[::-1]))) > 1e-3


def dense(a, b, c):
    K = len(b)
    A = np.diag(b)
    if K > 1:
        A += np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    return A


@pytest.mark.parametrize("K", [1, 2, 3, 5, 8, 16])
def test_thomas_vs_pivoted_dense_solve(orc, K):
    """B1: the oracle's Thomas solve agrees with LAPACK's partially pivoted LU
    (numpy.linalg.solve) within the condition-number bound."""
    f = fields(6, 5, K, 10 + K)
    for (i, j) in [(0, 0), (2, 3), (5, 4), (3, 1)]:
        a, b, c, d = orc.vadv_system(f["u_stage"], f["wcon"], f["u_pos"], f["utens"],
                                     f["utens_stage"], i, j)
        assert a[0] == 0.0 and c[-1] == 0.0
        x, piv, _ = orc.thomas(a, b, c, d)
        A = dense(a, b, c)
        xr = np.linalg.solve(A, d)
        kappa = np.linalg.cond(A, np.inf)
        growth = np.max(np.abs(piv)) / np.max(np.abs(b)) + np.max(np.abs(a[1:]) / np.abs(piv[:-1]), initial=1.0)
        bound = 50 * K * EPS * kappa * max(1.0, growth)
        assert np.max(np.abs(x - xr)) <= bound * np.max(np.abs(xr))


def exact_solve(a, b, c, d):
    """Gauss-Jordan elimination with exact rationals on the dense matrix (brute force)."""
    K = len(b)
    A = [[Fraction(0)] * K + [Fraction(d[r])] for r in range(K)]
    for r in range(K):
        A[r][r] = Fraction(b[r])
        if r > 0:
            A[r][r - 1] = Fraction(a[r])
        if r < K - 1:
            A[r][r + 1] = Fraction(c[r])
    for col in range(K):
        piv = next(r for r in range(col, K) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        for r in range(K):
            if r != col and A[r][col] != 0:
                m = A[r][col] / A[col][col]
                A[r] = [x - m * y for x, y in zip(A[r], A[col])]
    return [A[r][K] / A[r][r] for r in range(K)]


@pytest.mark.parametrize("K", [1, 2, 3, 4, 6])
def test_exact_rational_column(orc, K):
    """Brute force on tiny columns: dyadic inputs, the benchmark's coefficient set written out
    in exact rational arithmetic from its definition (a_k = -w_k/4, c_k = w_{k+1}/4,
    b_k = dtr - a_k - c_k, w the I-face average), solved exactly; the oracle output agrees to
    the binary64 rounding of the solve."""
    rng = np.random.default_rng(20 + K)
    I, J = 3, 2
    shp = (K, J + 2, I + 2)
    f = {n: rng.integers(-32, 32, shp) / 32.0 for n in ("u_stage", "u_pos", "utens", "utens_stage")}
    f["wcon"] = rng.integers(-16, 16, shp) / 32.0
    out = run(orc, f)
    dtr = Fraction(3, 20)
    for j in range(J):
        for i in range(I):
            col = lambda n: [Fraction(f[n][k, j + 1, i + 1]) for k in range(K)]
            us, up, ut, uts = col("u_stage"), col("u_pos"), col("utens"), col("utens_stage")
            w = [(Fraction(f["wcon"][k, j + 1, i + 1]) + Fraction(f["wcon"][k, j + 1, i + 2])) / 2
                 for k in range(K)]
            a = [Fraction(0) if k == 0 else -w[k] / 4 for k in range(K)]
            c = [Fraction(0) if k == K - 1 else w[k + 1] / 4 for k in range(K)]
            b = [dtr - a[k] - c[k] for k in range(K)]
            d = []
            for k in range(K):
                v = dtr * up[k] + ut[k] + uts[k]
                if k > 0:
                    v -= a[k] * (us[k - 1] - us[k])
                if k < K - 1:
                    v -= c[k] * (us[k + 1] - us[k])
                d.append(v)
            x = exact_solve(a, b, c, d)
            ref = np.array([float(dtr * (x[k] - up[k])) for k in range(K)])
            got = out[:, j + 1, i + 1]
            assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_binary64_vs_extended_thomas(orc):
    """B2: the binary64 solve stays within 1e-12 (max-norm relative, over many columns of the
    256x256x80 distributions) of the same recurrences carried in x87 extended precision."""
    f = fields(24, 24, 80, 30)
    err, ref = 0.0, 0.0
    for j in range(24):
        for i in range(24):
            a, b, c, d = orc.vadv_system(f["u_stage"], f["wcon"], f["u_pos"], f["utens"],
                                         f["utens_stage"], i, j)
            x, _, _ = orc.thomas(a, b, c, d)
            xl = orc.thomas(a, b, c, d, extended=True)
            err = max(err, np.max(np.abs(x - xl)))
            ref = max(ref, np.max(np.abs(xl)))
    assert err / ref < 1e-12


def test_lu_backward_error(orc):
    """R1: the computed solution satisfies |A x - d| <= 8u (|L||U||x|)_k row by row, L and U
    being the oracle's computed bidiagonal factors (l_k = a_k / p_{k-1}, U = (p, c)); the
    residual is evaluated in extended precision (no-pivoting LU backward error,
    Higham, Accuracy and Stability of Numerical Algorithms, Ch. 9)."""
    f = fields(16, 16, 80, 40)
    u = EPS / 2
    L = np.longdouble
    worst = 0.0
    for j in range(0, 16, 3):
        for i in range(16):
            a, b, c, d = orc.vadv_system(f["u_stage"], f["wcon"], f["u_pos"], f["utens"],
                                         f["utens_stage"], i, j)
            x, p, _ = orc.thomas(a, b, c, d)
            K = len(b)
            xa = x.astype(L)
            r = b.astype(L) * xa - d.astype(L)
            r[1:] += a[1:].astype(L) * xa[:-1]
            r[:-1] += c[:-1].astype(L) * xa[1:]
            l = np.zeros(K)
            l[1:] = a[1:] / p[:-1]
            # (|L||U||x|)_k = |l_k| (|p_{k-1}||x_{k-1}| + |c_{k-1}||x_k|) + |p_k||x_k| + |c_k||x_{k+1}|
            ux = np.abs(p) * np.abs(x)
            ux[:-1] += np.abs(c[:-1]) * np.abs(x[1:])
            lux = ux.copy()
            lux[1:] += np.abs(l[1:]) * ux[:-1]
            ratio = np.abs(r).astype(np.float64) / (u * lux)
            worst = max(worst, float(np.max(ratio)))
    assert worst <= 8.0, worst


def test_full_field_matches_column_solves(orc):
    """The field driver writes dtr*(x - u_pos) of each column's own solve."""
    f = fields(5, 4, 9, 50)
    out = run(orc, f)
    for (i, j) in [(0, 0), (4, 3), (2, 1)]:
        a, b, c, d = orc.vadv_system(f["u_stage"], f["wcon"], f["u_pos"], f["utens"],
                                     f["utens_stage"], i, j)
        x, _, _ = orc.thomas(a, b, c, d)
        assert np.array_equal(out[:, j + 1, i + 1], DTR * (x - f["u_pos"][:, j + 1, i + 1]))


def test_literal_wcon_mode_reads_one_face(orc):
    """wmode=1 reads wcon at i only: changing wcon at i+1 must not change the result."""
    f = fields(4, 3, 10, 60)
    out = run(orc, f, wmode=1)
    f["wcon"][:, :, 2:] += 0.01 * np.random.default_rng(61).uniform(-1, 1, f["wcon"][:, :, 2:].shape)
    g = dict(f)
    g["wcon"] = f["wcon"].copy()
    g["wcon"][:, 1:-1, 1] = fields(4, 3, 10, 60)["wcon"][:, 1:-1, 1]
    out2 = run(orc, g, wmode=1)
    assert np.array_equal(out[:, 1:-1, 1], out2[:, 1:-1, 1])


def test_beta_zero_equals_half_weights(orc):
    """beta_v enters only through the weights (1 +- beta)/2, which are exactly 1/2 at beta = 0;
    a nonzero beta_v moves weight between the implicit and explicit sides."""
    f = fields(6, 5, 20, 70, 0.15)
    base = run(orc, f)
    assert np.array_equal(base, run(orc, f, beta_v=0.0))
    assert np.max(np.abs(run(orc, f, beta_v=0.4) - base)) > 1e-6
