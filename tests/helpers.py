"""Shared helpers of the GPU parity tests: upload seeded inputs to padded
device storages, run the CUDA path through the C ABI, compare with the oracle.

Error metric (per output field, over the compute domain): max |gpu - oracle| /
max |oracle| (max-norm relative).  The worst column (max over a column of the
error divided by max over the column of |oracle|) is reported beside it."""
import numpy as np


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / (den if den > 0 else 1.0))


def worst_column(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.max(np.abs(got - ref), axis=0)
    den = np.maximum(np.max(np.abs(ref), axis=0), 1e-300)
    return float(np.max(num / den))


def region(a, origin, domain):
    (oi, oj, ok), (I, J, K) = origin, domain
    return a[ok:ok + K, oj:oj + J, oi:oi + I]


def s7_stats(got, ref, bound):
    """The secondary error statistics beside the max-norm (per output field, over the
    domain): the worst column's relative error, the 99.9th percentile of the pointwise
    relative error |gpu - oracle| / |oracle| (a point where the oracle is 0 counts 0 if
    the GPU is 0 too, else infinity) and the fraction of points whose pointwise relative
    error exceeds `bound`."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(got - ref)
    a = np.abs(ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        pw = np.where(a > 0, d / np.where(a > 0, a, 1.0), np.where(d > 0, np.inf, 0.0))
    return {"max_norm": rel_err(got, ref), "worst_column": worst_column(got, ref),
            "p99_9_pointwise": float(np.percentile(pw, 99.9)), "frac_beyond": float(np.mean(pw > bound))}


def hdiff_point_bound(out_ref, inp, coeff, origin, domain):
    """The per-point bound of the binary64 hdiff against the binary64 oracle:
        |gpu - oracle|(i,j,k) <= 2^-51 |out(i,j,k)| + (2^-53 + 2^-43 |coeff(i,j,k)|) M(k),
    M(k) = the largest |in| over level k of the storage.  The GPU forms the Laplacian ->
    flux -> divergence chain exactly in int64 fixed point with unit 2^(E-1078), E the
    largest binary64 exponent its strip (or tile) reads at that level, so every input is
    truncated by less than 2^-55 M(k) and D (whose 13-point weights sum to at most 64 in
    magnitude) by less than 2^-49 M(k); the oracle rounds each of its lap, flux and
    divergence operations (at most 46 half-units of 2^-53 M(k) in D, about 2^-44.5 M(k)).
    A limiter decision can differ between the two only where the flux is within the
    oracle's own rounding of zero.  Both round the final out once (2^-53 |out| each) and
    the product coeff * D once.  Every term is covered by the coeff-scaled part (D's
    errors times |coeff|, < 2^-44 |coeff| M(k) together), the 2^-53 M(k) part (the
    truncation of in itself when the update runs in fixed point) and the |out| part."""
    (oi, oj, ok), (I, J, K) = origin, domain
    M = np.max(np.abs(inp[ok:ok + K]), axis=(1, 2))[:, None, None]
    c = np.abs(coeff[ok:ok + K, oj:oj + J, oi:oi + I])
    return 2.0 ** -51 * np.abs(out_ref) + (2.0 ** -53 + 2.0 ** -43 * c) * M
