"""torch.autograd.Function over gpcg_n1_adjoint.

``N1OverloadLoss.apply(ctx_obj, outages, P, b)`` returns the scalar overload
penalty summed over the N-1 scenarios (DC model); its backward multiplies
the library's adjoint gradients dL/dP and dL/db by the incoming gradient.
The library computes loss and both gradients in one call (forward); backward
only scales them.
"""
from __future__ import annotations

import torch


class N1OverloadLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, solver, outages, P, b):
        P = P.detach().to(torch.float64).contiguous()
        b = b.detach().to(torch.float64).contiguous()
        loss = torch.zeros(1, dtype=torch.float64, device=P.device)
        gP = torch.zeros_like(P)
        gb = torch.zeros_like(b)
        if P.is_cuda:
            solver.n1_adjoint_device(outages.to(torch.int32).contiguous(), P, b, loss, gP, gb)
        else:
            L, a, c = solver.n1_adjoint(outages.cpu().numpy(), P.numpy(), b.numpy())
            loss[0] = L
            gP.copy_(torch.from_numpy(a))
            gb.copy_(torch.from_numpy(c))
        fctx.save_for_backward(gP, gb)
        return loss[0]

    @staticmethod
    def backward(fctx, grad_out):
        gP, gb = fctx.saved_tensors
        return None, None, grad_out * gP, grad_out * gb
