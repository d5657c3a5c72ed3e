"""torch.autograd.Function over the library's log-joint adjoint (bmf_logjoint_grad).

The forward pass calls the CUDA adjoint once, which returns the value and the gradients with
respect to X, W and log alpha; backward scales the saved gradients by the incoming gradient.
Argument marshalling only: all arithmetic runs in libbmf."""
from __future__ import annotations

import torch


class LogJoint(torch.autograd.Function):
    """value = LogJoint.apply(ctx_bmf, subset, X, W, log_alpha): X [n, ld], W [d, ld] CUDA float32
    (ld % 4 == 0, padding ignored), log_alpha a 0-d float64 tensor.  Returns a 0-d float64
    tensor on X's device."""

    @staticmethod
    def forward(fctx, model, subset, X, W, log_alpha):
        X = X.contiguous()
        W = W.contiguous()
        if X.dtype != torch.float32 or W.dtype != torch.float32 or not X.is_cuda:
            raise TypeError("X and W must be CUDA float32 tensors")
        gX = torch.empty_like(X)
        gW = torch.empty_like(W)
        value, g_la = model.logjoint_grad(int(subset), X.data_ptr(), W.data_ptr(), X.shape[1],
                                          float(log_alpha), gX.data_ptr(), gW.data_ptr())
        fctx.save_for_backward(gX, gW)
        fctx.g_la = g_la
        return torch.tensor(value, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(fctx, g):
        gX, gW = fctx.saved_tensors
        gf = g.to(torch.float32)
        g_la = torch.as_tensor(fctx.g_la, dtype=torch.float64, device=g.device) * g
        return None, None, gX * gf, gW * gf, g_la
