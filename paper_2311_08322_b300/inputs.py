"""Seeded synthetic inputs for the hdiff / vadv workloads.

This module is the one piece shared by the CUDA path and the CPU oracle: it
draws random storages and nothing else (no stencil arithmetic).  Every field
is a whole storage, halo included, as a C-ordered float64 numpy array shaped
``(nk, nj, ni)`` (i fastest), drawn with ``numpy.random.default_rng(seed)``
(PCG64) in a fixed order.  Reduced-precision workloads round these float64
draws to float32 (``astype``), so both sides see identical values.

Workload shapes follow the benchmark set of the GT4Py paper (Sec. 3.1: a
horizontal-diffusion and a vertical-advection stencil on 3-D fields with
halos); the paper prints no sizes, so the sizes below are the library's own:
  * hdiff 64x64x40 FP64, halo 2 (storage 68x68x40): in ~ U(-1,1), coeff ~ U(0,0.025)
  * hdiff + vadv 256x256x80 FP64 (hdiff halo 2, vadv halo 1 in I/J):
    u_stage, u_pos, utens, utens_stage ~ U(-1,1), wcon ~ U(-0.5,0.5)
  * the same generators at 512x512x80 rounded to FP32
  * a 48-member ensemble of uneven domains (I=J in {48,96,128,192,256,384},
    K in {40,60,80,137})
  * a 10-step chain at 256x256x80 whose wcon is drawn from U(-0.3,0.3)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HDIFF_HALO = 2
VADV_HALO = 1
HDIFF_FIELDS = ("in", "coeff")
VADV_FIELDS = ("u_stage", "u_pos", "utens", "utens_stage", "wcon")


def storage_shape(I: int, J: int, K: int, halo: int) -> tuple:
    """(nk, nj, ni) of a storage with an I/J halo of ``halo`` points (none in K)."""
    return (K, J + 2 * halo, I + 2 * halo)


def hdiff_fields(rng: np.random.Generator, I: int, J: int, K: int, halo: int = HDIFF_HALO) -> dict:
    """``in`` then ``coeff``, both over the whole halo-``halo`` storage."""
    shp = storage_shape(I, J, K, halo)
    return {"in": rng.uniform(-1.0, 1.0, shp), "coeff": rng.uniform(0.0, 0.025, shp)}


def vadv_fields(rng: np.random.Generator, I: int, J: int, K: int, halo: int = VADV_HALO,
                wcon_amp: float = 0.5) -> dict:
    """``u_stage, u_pos, utens, utens_stage, wcon`` in that order, over the halo-1 storage."""
    shp = storage_shape(I, J, K, halo)
    out = {}
    for name in ("u_stage", "u_pos", "utens", "utens_stage"):
        out[name] = rng.uniform(-1.0, 1.0, shp)
    out["wcon"] = rng.uniform(-wcon_amp, wcon_amp, shp)
    return out


def hdiff_small(seed: int = 0) -> dict:
    """hdiff FP64 at 64x64x40 (storage 68x68x40)."""
    return hdiff_fields(np.random.default_rng(seed), 64, 64, 40)


def hdiff_vadv(I: int = 256, J: int = 256, K: int = 80, seed: int = 0, wcon_amp: float = 0.5) -> dict:
    """hdiff fields then vadv fields from one generator (FP64 draws)."""
    rng = np.random.default_rng(seed)
    d = hdiff_fields(rng, I, J, K)
    d.update(vadv_fields(rng, I, J, K, wcon_amp=wcon_amp))
    return d


def to_f32(fields: dict) -> dict:
    """Round every float64 draw to float32 (the reduced-precision workloads)."""
    return {k: v.astype(np.float32) for k, v in fields.items()}


@dataclass
class Member:
    I: int
    J: int
    K: int
    seed: int
    fields: dict = field(default_factory=dict, repr=False)


ENSEMBLE_IJ = (48, 96, 128, 192, 256, 384)
ENSEMBLE_K = (40, 60, 80, 137)


def ensemble_shapes(n_members: int = 48, seed: int = 0) -> list:
    """Uneven member domains: I=J uniform over ENSEMBLE_IJ, K uniform over ENSEMBLE_K."""
    rng = np.random.default_rng(seed)
    ij = rng.choice(ENSEMBLE_IJ, size=n_members)
    kk = rng.choice(ENSEMBLE_K, size=n_members)
    return [(int(a), int(a), int(b)) for a, b in zip(ij, kk)]


def ensemble(n_members: int = 48, seed: int = 0, dtype=np.float32, materialize: bool = True) -> list:
    """Members with their hdiff + vadv fields (member m drawn from seed ``seed*1000 + 1 + m``)."""
    out = []
    for m, (I, J, K) in enumerate(ensemble_shapes(n_members, seed)):
        mem = Member(I, J, K, seed * 1000 + 1 + m)
        if materialize:
            f = hdiff_vadv(I, J, K, seed=mem.seed)
            mem.fields = {k: v.astype(dtype) for k, v in f.items()}
        out.append(mem)
    return out


def chain_inputs(I: int = 256, J: int = 256, K: int = 80, seed: int = 0, wcon_amp: float = 0.3) -> dict:
    """10-step chain: initial field + coeff (halo 2), then the fixed vadv inputs."""
    return hdiff_vadv(I, J, K, seed=seed, wcon_amp=wcon_amp)
