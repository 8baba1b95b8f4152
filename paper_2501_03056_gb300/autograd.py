"""torch.autograd.Function for the uniformity energy (hand-written backward).

E(y, verts) = sum over mobile particles of (rho_i - W0)^2 at positions
x = P(y): surface particles projected onto the plane of their current
(frozen) triangle built from ``verts``, all others x = y.  Forward and
backward are the library's CUDA kernels (``fppg_energy``); torch only holds
the device buffers and the stream.
"""
from __future__ import annotations

import torch

from . import Body


class UniformityEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y: torch.Tensor, verts: torch.Tensor, body: Body):
        if not (y.is_cuda and verts.is_cuda):
            raise ValueError("UniformityEnergy runs on the GPU only")
        y = y.detach().contiguous().float()
        verts = verts.detach().contiguous().float()
        body.set_stream(torch.cuda.current_stream())
        E = body.energy_ptr(y.data_ptr(), verts.data_ptr())
        ctx.save_for_backward(y, verts)
        ctx.body = body
        return torch.tensor(E, dtype=torch.float64, device=y.device)

    @staticmethod
    def backward(ctx, gE):
        y, verts = ctx.saved_tensors
        gy = torch.empty_like(y)
        gV = torch.empty_like(verts)
        ctx.body.set_stream(torch.cuda.current_stream())
        ctx.body.energy_ptr(y.data_ptr(), verts.data_ptr(), gy.data_ptr(), gV.data_ptr())
        s = gE.to(torch.float32)
        return gy * s, gV * s, None


def uniformity_energy(y: torch.Tensor, verts: torch.Tensor, body: Body) -> torch.Tensor:
    return UniformityEnergy.apply(y, verts, body)
