"""The windowed cost as a torch.autograd.Function.

Forward and backward are the C ABI's window kernels (prost_window_eval): the
forward writes the cost, the backward runs the pass again and writes dF/dU,
dF/dY and dF/dmu multiplied by the upstream gradient inside the kernel, so no
arithmetic of the method runs in PyTorch, which only supplies device memory.
"""

from __future__ import annotations

from . import prost as _p

_FN = None


def _autograd_fn():
    global _FN
    if _FN is not None:
        return _FN
    import torch

    class WindowFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, U, Y, mu, X, labels, win):
            for t in (U, Y, mu, X):
                if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                    raise ValueError("U, Y, mu and X must be contiguous float32 CUDA tensors")
            cost = torch.empty((), dtype=torch.float32, device=U.device)
            _p.prost_window_eval(win.handle, U, Y, X, labels, mu, cost)
            ctx.win = win
            ctx.labels = labels
            ctx.save_for_backward(U, Y, mu, X)
            return cost

        @staticmethod
        def backward(ctx, g):
            U, Y, mu, X = ctx.saved_tensors
            g = g.contiguous()
            dU = torch.empty_like(U)
            dY = torch.empty_like(Y)
            dmu = torch.empty_like(mu)
            cost = torch.empty((), dtype=torch.float32, device=U.device)
            _p.prost_window_eval(ctx.win.handle, U, Y, X, ctx.labels, mu, cost, dU, dY, dmu, gscale=g)
            return dU, dY, dmu, None, None, None

    _FN = WindowFn
    return _FN


class WindowCost:
    """The cost over a window of n frames of m entries (channels x pixels)
    for a rank-k subspace: call it with (U m x k, Y k x n, mu (0-d), X n x m,
    labels n x pixels or None) for a differentiable cost."""

    def __init__(self, m, channels, k, n, p=0.25, omega=5e-5, stream=None):
        self.m, self.channels, self.k, self.n = m, channels, k, n
        self.handle = _p.prost_window_init(m, channels, k, n, p, omega, stream)

    def close(self):
        if getattr(self, "handle", None):
            _p.prost_window_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def __call__(self, U, Y, mu, X, labels=None):
        return _autograd_fn().apply(U, Y, mu, X, labels, self)

    def ustep(self, U, dU, t, U_out, status_out=None):
        """U_out = Cholesky-QR retraction of U - t (I - U U^T) dU (device tensors)."""
        return _p.prost_window_ustep(self.handle, U, dU, t, U_out, status_out)
