"""torch.autograd.Function over the C-ABI adjoint (argument marshalling only).

``SFSegPower.apply(sp, f, x0, engine, iters)`` returns x^K of ``iters``
normalised power steps; its backward calls ``sfseg_adjoint`` (the hand-written
reverse mode of the unrolled iteration, with checkpointed recomputation) and
returns dL/dsp, dL/df, dL/dx0.  ``engine`` is an ``SFSeg`` created with
``flags = SFSEG_RECORD | SFSEG_S_IS_SP`` for the volume's shape; sp = S^p and
any other preprocessing are ordinary torch operations around this function.
"""
from __future__ import annotations

import torch

from . import SFSEG_RECORD, SFSEG_S_IS_SP, SFSeg


class SFSegPower(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sp, f, x0, engine: SFSeg, iters: int):
        if not (engine.params.flags & SFSEG_RECORD and engine.params.flags & SFSEG_S_IS_SP):
            raise ValueError("engine needs flags SFSEG_RECORD | SFSEG_S_IS_SP")
        ctx.engine = engine
        return engine.power_iterate(sp.detach().contiguous(), f.detach().contiguous(),
                                    x0.detach().contiguous(), iters)

    @staticmethod
    def backward(ctx, gx):
        gsp, gf, gx0 = ctx.engine.adjoint(gx.contiguous())
        return gsp, gf, gx0, None, None


def make_engine(shape, **kw) -> SFSeg:
    """SFSeg engine set up for SFSegPower (recording, sp passed directly)."""
    flags = kw.pop("flags", 0) | SFSEG_RECORD | SFSEG_S_IS_SP
    return SFSeg(shape, flags=flags, **kw)
