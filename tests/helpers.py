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
