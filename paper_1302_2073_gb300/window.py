"""The windowed cost as a torch.autograd.Function.

The forward is the C ABI's window kernel (prost_window_eval).  When an input
needs a gradient, that one pass also writes dF/dU, dF/dY and dF/dmu (the
hand-written adjoint), which the backward only scales by the upstream
gradient; otherwise the pass writes the cost alone.  No arithmetic of the
method runs in PyTorch, which supplies device memory and the scaling.
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
            if any(ctx.needs_input_grad[:3]):
                dU, dY, dmu = torch.empty_like(U), torch.empty_like(Y), torch.empty_like(mu)
                _p.prost_window_eval(win.handle, U, Y, X, labels, mu, cost, dU, dY, dmu)
                ctx.save_for_backward(dU, dY, dmu)
            else:
                _p.prost_window_eval(win.handle, U, Y, X, labels, mu, cost)
            return cost

        @staticmethod
        def backward(ctx, g):
            dU, dY, dmu = ctx.saved_tensors
            return (dU * g if ctx.needs_input_grad[0] else None, dY * g if ctx.needs_input_grad[1] else None,
                    dmu * g if ctx.needs_input_grad[2] else None, None, None, None)

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
