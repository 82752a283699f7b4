"""Differentiable chained hdiff -> vadv steps (torch.autograd) on libgtb.

One step of the chain, on a periodic (I, J) domain of K levels:
    field storage <- field (interior, halo refreshed periodically, 2 points)
    h             <- hdiff(field, coeff)
    field'        <- vadv(u_stage = h, u_pos = h, utens, utens_stage, wcon)
utens, utens_stage and wcon are fixed inputs of every step.  The forward runs
the two stencils as one kernel (gtb_hdiff_vadv: h never leaves the chip).  The step's
backward runs the hand-written adjoint kernels (gtb_vadv_adj with the u_stage
and u_pos cotangents merged, gtb_hdiff_adj with the limiter recomputed from
the saved input, gtb_halo_periodic_adj) — no autodiff of the stencils.  Each
step saves its input field (step-level checkpointing: an N-step chain holds N
field copies) and, unless ChainFixed.save_factors is off, the factors of its
column solves, which the vadv adjoint then reads instead of refactorising.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import gtb


@dataclass
class ChainFixed:
    """Fixed inputs of every step: wcon (halo 1 in I), utens and utens_stage (interior)."""
    wcon: gtb.Storage
    utens: gtb.Storage
    utens_stage: gtb.Storage
    dtr_stage: float = 3.0 / 20.0
    beta_v: float = 0.0
    # keep each step's column factors (c'_k, 1/p_k: two K x I x J arrays) so that the backward
    # does not refactorise A: memory for FP64-pipe time
    save_factors: bool = True

    @property
    def prec(self):
        return "native" if self.utens.data.dtype == torch.float64 else "df"


def interior_storage(I, J, K, dtype, device="cuda"):
    return gtb.Storage(gtb.empty_storage(I, J, K, dtype=dtype, device=device), (0, 0, 0))


def halo_storage(I, J, K, dtype, halo=2, device="cuda"):
    return gtb.Storage(gtb.empty_storage(I + 2 * halo, J + 2 * halo, K, dtype=dtype, device=device, halo_i=halo),
                       (halo, halo, 0))


def _as_storage(t: torch.Tensor) -> gtb.Storage:
    """An interior tensor (K, J, I) as a storage with origin 0 (copied into the padded layout)."""
    K, J, I = t.shape
    s = interior_storage(I, J, K, t.dtype, t.device)
    s.data.copy_(t)
    return s


class ChainStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field: torch.Tensor, coeff: torch.Tensor, fixed: ChainFixed):
        K, J, I = field.shape
        fs = halo_storage(I, J, K, field.dtype, 2, field.device)
        fs.interior((I, J, K)).copy_(field)
        gtb.halo_periodic(fs, 2, 2, domain=(I, J, K))
        cs = _as_storage(coeff)
        y = interior_storage(I, J, K, field.dtype, field.device)
        # h = hdiff(field, coeff) and y = vadv(h, wcon, h, utens, utens_stage) in one kernel
        # (h stays on chip; the backward needs only the checkpointed input and, if kept, the factors)
        ws = "auto"
        if fixed.save_factors:
            nb = gtb.hdiff_vadv_workspace_bytes(field.dtype, fixed.prec, (I, J, K), save_factors=True)
            ws = torch.empty(nb, dtype=torch.uint8, device=field.device)
        gtb.hdiff_vadv(fs, cs, fixed.wcon, fixed.utens, fixed.utens_stage, y, dtr_stage=fixed.dtr_stage,
                       beta_v=fixed.beta_v, prec=fixed.prec, domain=(I, J, K), workspace=ws,
                       save_factors=fixed.save_factors)
        ctx.fixed = fixed
        ctx.fs, ctx.cs = fs, cs  # the checkpoint: this step's input (with its halo) and coeff
        ctx.factors = ws if fixed.save_factors else None
        return y.data.clone()

    @staticmethod
    def backward(ctx, y_bar: torch.Tensor):
        fixed, fs, cs = ctx.fixed, ctx.fs, ctx.cs
        K, J, I = y_bar.shape
        yb = _as_storage(y_bar.contiguous())
        hb = interior_storage(I, J, K, y_bar.dtype, y_bar.device)
        # h entered vadv as both u_stage and u_pos: one merged cotangent
        if ctx.factors is not None:  # the forward's factors (consumed)
            gtb.vadv_adj(fixed.wcon, yb, hb, hb, dtr_stage=fixed.dtr_stage, beta_v=fixed.beta_v, prec=fixed.prec,
                         domain=(I, J, K), workspace=ctx.factors, factors=True)
            ctx.factors = None
        else:
            gtb.vadv_adj(fixed.wcon, yb, hb, hb, dtr_stage=fixed.dtr_stage, beta_v=fixed.beta_v, prec=fixed.prec,
                         domain=(I, J, K))
        ib = halo_storage(I, J, K, y_bar.dtype, 2, y_bar.device)
        cb = interior_storage(I, J, K, y_bar.dtype, y_bar.device)
        gtb.hdiff_adj(fs, cs, hb, ib, cb, domain=(I, J, K))
        gtb.halo_periodic_adj(ib, 2, 2, domain=(I, J, K))
        field_bar = ib.interior((I, J, K)).clone() if ctx.needs_input_grad[0] else None
        coeff_bar = cb.data.clone() if ctx.needs_input_grad[1] else None
        return field_bar, coeff_bar, None


def chain(field: torch.Tensor, coeff: torch.Tensor, fixed: ChainFixed, steps: int = 10) -> torch.Tensor:
    """`steps` chained steps; differentiable in field and coeff."""
    for _ in range(steps):
        field = ChainStep.apply(field, coeff, fixed)
    return field


def chain_inputs(I=256, J=256, K=80, seed=0, dtype=torch.float64, wcon_amp=0.3, device="cuda"):
    """Initial field and coeff (interior tensors) and the fixed vadv inputs, from the seeded
    generators (the 10-step chain draws wcon from U(-0.3, 0.3))."""
    from . import inputs
    import numpy as np
    f = inputs.chain_inputs(I, J, K, seed=seed, wcon_amp=wcon_amp)
    npd = np.float64 if dtype == torch.float64 else np.float32
    field = torch.from_numpy(np.ascontiguousarray(f["in"][:, 2:-2, 2:-2].astype(npd))).to(device)
    coeff = torch.from_numpy(np.ascontiguousarray(f["coeff"][:, 2:-2, 2:-2].astype(npd))).to(device)
    fixed = ChainFixed(wcon=gtb.storage_from(f["wcon"].astype(npd), (1, 1, 0), device=device),
                       utens=gtb.storage_from(np.ascontiguousarray(f["utens"][:, 1:-1, 1:-1].astype(npd)), (0, 0, 0),
                                              device=device),
                       utens_stage=gtb.storage_from(np.ascontiguousarray(f["utens_stage"][:, 1:-1, 1:-1].astype(npd)),
                                                    (0, 0, 0), device=device))
    return field, coeff, fixed, f
