"""The synthetic video recipe of ``video.py`` generated on the GPU with torch.

Long measurement runs (thousands of 1080p frames, or a tick of 64 streams)
need frames far faster than numpy makes them.  :class:`DeviceVideo` takes a
:class:`SyntheticVideo` and produces its frames on the device: the planted
subspace, the coefficient walk and the moving shapes are the host stream's
own (so the background and the ground truth are identical), while the per-frame
draws (foreground values, jitter, noise) come from torch's generator seeded by
(seed, t).  Frames are therefore reproducible but not bit-equal to the numpy
ones; where a test compares against the oracle frame by frame, it uses the
numpy stream.  Input generation only: nothing of pROST's arithmetic is here.
"""

from __future__ import annotations

import math

import numpy as np

from .video import SyntheticVideo, _reflect


class DeviceVideo:
    """Frames of ``vid`` generated on ``device`` (see the module docstring)."""

    def __init__(self, vid: SyntheticVideo, device):
        import torch
        self.torch = torch
        self.vid = vid
        self.device = torch.device(device)
        self.U0 = torch.from_numpy(vid.U0.astype(np.float32)).to(self.device)
        self.Y0 = torch.from_numpy(vid.Y0.astype(np.float32)).to(self.device)
        self.xs = torch.arange(vid.width, dtype=torch.float32, device=self.device) + 0.5
        self.ys = torch.arange(vid.height, dtype=torch.float32, device=self.device) + 0.5
        self.gen = torch.Generator(device=self.device)

    def shape_mask(self, t: int):
        v, torch = self.vid, self.torch
        fg = torch.zeros((v.height, v.width), dtype=torch.bool, device=self.device)
        for s in v.shapes:
            cx = _reflect(s.x0, s.vx, t, s.hx, v.width - s.hx)
            cy = _reflect(s.y0, s.vy, t, s.hy, v.height - s.hy)
            if s.kind == "rect":
                fg |= ((self.ys - cy).abs() <= s.hy)[:, None] & ((self.xs - cx).abs() <= s.hx)[None, :]
            else:
                dx = ((self.xs - cx) / s.hx) ** 2
                dy = ((self.ys - cy) / s.hy) ** 2
                fg |= (dy[:, None] + dx[None, :]) <= 1.0
        return fg

    def frame(self, t: int, out=None):
        """Frame t as a (C, H, W) device tensor (uint8 or float32), written
        into ``out`` when given."""
        v, torch = self.vid, self.torch
        self.gen.manual_seed(int(v.seed) * 1_000_003 + int(t) + 1)
        b = v.offset + v.scale * (self.U0 @ self.Y0[t])
        x = b.reshape(v.channels, v.height, v.width)
        fg = self.shape_mask(t)
        u = torch.rand(x.shape, generator=self.gen, device=self.device)
        x = torch.where(fg[None], u, x)
        if v.jitter:
            d = torch.randint(-v.jitter, v.jitter + 1, (2,), generator=self.gen, device=self.device).tolist()
            rows = (torch.arange(v.height, device=self.device) - d[1]).clamp(0, v.height - 1)
            cols = (torch.arange(v.width, device=self.device) - d[0]).clamp(0, v.width - 1)
            x = x[:, rows][:, :, cols]
        x = x + v.noise_sigma * torch.randn(x.shape, generator=self.gen, device=self.device)
        x = x.clamp_(0.0, 1.0)
        if v.dtype == "u8":
            x = torch.round(255.0 * x).to(torch.uint8)
        if out is not None:
            out.copy_(x)
            return out
        return x.contiguous()
