"""Seeded synthetic video: random-walk low-rank background + moving foreground + noise.

Recipe (stands in for the real surveillance videos of the paper's evaluation,
Section 5, which are not used here):

* planted subspace ``U0``: orthonormal factor of a seeded Gaussian m x k matrix;
* coefficients ``y_0 ~ N(0, I_k)``, ``y_t = y_{t-1} + walk_sigma * N(0, I_k)``;
* background ``b_t = offset + amplitude * sqrt(m/k) * U0 y_t`` (per-entry std
  close to ``amplitude``), entries stacked channel-planar as in Section 3.4;
* foreground: ``n_shapes`` axis-aligned rectangles or ellipses of total area
  ``fg_fraction`` of the image, moving with integer velocities of 1-3 px per
  frame and reflecting at the borders; inside them every channel is replaced by
  i.i.d. U(0, 1);
* optional camera jitter: the whole composed frame (and its ground truth)
  shifted by a uniform integer (dx, dy) in [-J, J]^2 with edge replication;
* additive N(0, noise_sigma^2), clip to [0, 1], and for uint8 frames
  ``round(255 v)``.

Every frame is generated from its own PCG64 stream keyed by (seed, t), so a
frame can be produced at random, and the same frame is produced on any machine.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def random_orthonormal(m: int, k: int, rng) -> np.ndarray:
    """Orthonormal m x k matrix: Q of a reduced QR of a Gaussian matrix,
    columns signed so that diag(R) > 0 (makes the result unique)."""
    if not isinstance(rng, np.random.Generator):
        rng = np.random.Generator(np.random.PCG64(rng))
    g = rng.standard_normal((m, k))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.ascontiguousarray(q * s)


@dataclass
class _Shape:
    kind: str
    x0: float
    y0: float
    hx: float  # half extent along x
    hy: float  # half extent along y
    vx: int
    vy: int


def _reflect(p0: float, v: int, t: int, lo: float, hi: float) -> float:
    """Position after t frames of constant velocity v, reflecting in [lo, hi]."""
    span = hi - lo
    if span <= 0:
        return lo
    u = (p0 - lo + v * t) % (2.0 * span)
    return lo + (u if u <= span else 2.0 * span - u)


class SyntheticVideo:
    """One seeded synthetic camera stream (see module docstring for the recipe)."""

    def __init__(self, width: int, height: int, channels: int = 1, k: int = 5,
                 n_frames: int = 200, fg_fraction: float = 0.05, shape: str = "rect",
                 n_shapes: int = 3, jitter: int = 0, noise_sigma: float = 0.01,
                 walk_sigma: float = 0.02, amplitude: float = 0.1, offset: float = 0.5,
                 seed: int = 0, dtype: str = "u8"):
        if shape not in ("rect", "ellipse"):
            raise ValueError("shape must be 'rect' or 'ellipse'")
        if dtype not in ("u8", "f32"):
            raise ValueError("dtype must be 'u8' or 'f32'")
        self.width, self.height, self.channels = int(width), int(height), int(channels)
        self.P = self.width * self.height
        self.m = self.channels * self.P
        self.k, self.n_frames = int(k), int(n_frames)
        self.fg_fraction, self.shape, self.n_shapes = float(fg_fraction), shape, int(n_shapes)
        self.jitter, self.noise_sigma = int(jitter), float(noise_sigma)
        self.walk_sigma, self.amplitude, self.offset = float(walk_sigma), float(amplitude), float(offset)
        self.seed, self.dtype = int(seed), dtype

        rng = np.random.Generator(np.random.PCG64(self.seed))
        self.U0 = random_orthonormal(self.m, self.k, rng)
        steps = rng.standard_normal((self.n_frames, self.k))
        steps[1:] *= self.walk_sigma
        self.Y0 = np.cumsum(steps, axis=0)  # y_0 ~ N(0, I), then a Gaussian random walk
        self.scale = self.amplitude * math.sqrt(self.m / self.k)

        self.shapes = []
        area = self.fg_fraction * self.P / max(self.n_shapes, 1)
        for _ in range(self.n_shapes if self.fg_fraction > 0 else 0):
            aspect = rng.uniform(0.5, 2.0)
            if shape == "rect":
                w = math.sqrt(area * aspect)
                h = area / w
                hx, hy = w / 2.0, h / 2.0
            else:
                a = math.sqrt(area * aspect / math.pi)
                hx, hy = a, area / (math.pi * a)
            hx = min(hx, self.width / 2.0)
            hy = min(hy, self.height / 2.0)
            x0 = rng.uniform(hx, self.width - hx)
            y0 = rng.uniform(hy, self.height - hy)
            speeds = np.array([-3, -2, -1, 1, 2, 3])
            vx, vy = (int(v) for v in rng.choice(speeds, size=2))
            self.shapes.append(_Shape(shape, x0, y0, hx, hy, vx, vy))
        self._xs = np.arange(self.width, dtype=np.float64) + 0.5
        self._ys = np.arange(self.height, dtype=np.float64) + 0.5

    # -- pieces ---------------------------------------------------------------
    def shape_mask(self, t: int) -> np.ndarray:
        """(H, W) bool: pixels covered by the moving shapes at frame t (before jitter)."""
        fg = np.zeros((self.height, self.width), dtype=bool)
        for s in self.shapes:
            cx = _reflect(s.x0, s.vx, t, s.hx, self.width - s.hx)
            cy = _reflect(s.y0, s.vy, t, s.hy, self.height - s.hy)
            if s.kind == "rect":
                cols = np.abs(self._xs - cx) <= s.hx
                rows = np.abs(self._ys - cy) <= s.hy
                fg |= rows[:, None] & cols[None, :]
            else:
                dx = ((self._xs - cx) / s.hx) ** 2
                dy = ((self._ys - cy) / s.hy) ** 2
                fg |= (dy[:, None] + dx[None, :]) <= 1.0
        return fg

    def background(self, t: int) -> np.ndarray:
        """(C, H, W) float64 noiseless background of frame t."""
        b = self.offset + self.scale * (self.U0 @ self.Y0[t])
        return b.reshape(self.channels, self.height, self.width)

    def _shift(self, a: np.ndarray, dx: int, dy: int) -> np.ndarray:
        rows = np.clip(np.arange(self.height) - dy, 0, self.height - 1)
        cols = np.clip(np.arange(self.width) - dx, 0, self.width - 1)
        return a[..., rows, :][..., :, cols]

    # -- frames ---------------------------------------------------------------
    def frame(self, t: int):
        """Frame t as ((C, H, W) uint8 or float32 array, (H, W) bool ground-truth mask)."""
        if not 0 <= t < self.n_frames:
            raise IndexError(f"frame {t} outside [0, {self.n_frames})")
        frng = np.random.Generator(np.random.PCG64([self.seed, 1, int(t)]))
        v = self.background(t)
        fg = self.shape_mask(t)
        n_fg = int(fg.sum())
        if n_fg:
            v[:, fg] = frng.random((self.channels, n_fg))
        if self.jitter:
            dx, dy = (int(d) for d in frng.integers(-self.jitter, self.jitter + 1, size=2))
            v = self._shift(v, dx, dy)
            fg = self._shift(fg, dx, dy)
        v += self.noise_sigma * frng.standard_normal(v.shape)
        np.clip(v, 0.0, 1.0, out=v)
        if self.dtype == "u8":
            out = np.rint(255.0 * v).astype(np.uint8)
        else:
            out = v.astype(np.float32)
        return np.ascontiguousarray(out), np.ascontiguousarray(fg)

    def frames(self, start: int, count: int) -> np.ndarray:
        """(count, C, H, W) stack of frames start .. start+count-1."""
        first, _ = self.frame(start)
        out = np.empty((count,) + first.shape, dtype=first.dtype)
        out[0] = first
        for i in range(1, count):
            out[i], _ = self.frame(start + i)
        return out


# pROST parameters of the paper's benchmark run (Section 5.1): k=15, omega=5e-5,
# t_init=5e-3, t_min=1e-4, delta=0.35, p=0.25, mu=delta^2(1-p), <=5 CG steps.
# The step sizes were chosen for 160x120 RGB frames (m = 57,600); the projected
# gradient norm times |y| grows in proportion to m for the same per-entry data,
# so larger frames scale t_init and t_min by 57,600/m to keep the geodesic angle
# in the same range (both stay inside the ranges of Section 3.4).
_PAPER = dict(p=0.25, delta=0.35, mu=0.091875, omega=5e-5, t_init=5e-3, t_min=1e-4,
              i_init=100, n_cg=5)


def _params(m: int, k: int, dtype: str, **over):
    prm = dict(_PAPER)
    prm["k"] = k
    s = min(1.0, 57600.0 / m)
    prm["t_init"] *= s
    prm["t_min"] *= s
    prm["in_scale"] = 1.0 / 255.0 if dtype == "u8" else 1.0
    prm["in_offset"] = 0.5
    prm.update(over)
    return prm


# Workloads: the sizes, value distributions and structure of the paper's
# streams, at the resolutions the measurements use.
WORKLOADS = {
    "gray160x120_k5": dict(
        video=dict(width=160, height=120, channels=1, k=5, n_frames=200, fg_fraction=0.05,
                   shape="rect", n_shapes=3, jitter=0, seed=1000, dtype="f32")),
    "rgb640x480_k10": dict(
        video=dict(width=640, height=480, channels=3, k=10, n_frames=1000, fg_fraction=0.08,
                   shape="ellipse", n_shapes=3, jitter=2, seed=2000, dtype="u8")),
    "rgb1920x1080_k15": dict(
        video=dict(width=1920, height=1080, channels=3, k=15, n_frames=2000, fg_fraction=0.10,
                   shape="ellipse", n_shapes=3, jitter=3, seed=5000, dtype="u8")),
}


def make_workload(name: str, **video_over):
    """(SyntheticVideo, pROST parameter dict) of a named workload."""
    spec = WORKLOADS[name]
    vkw = dict(spec["video"])
    vkw.update(video_over)
    vid = SyntheticVideo(**vkw)
    prm = _params(vid.m, vid.k, vid.dtype)
    prm.update(width=vid.width, height=vid.height, channels=vid.channels,
               frame_dtype=vid.dtype)
    return vid, prm


# Many streams of uneven size and rank advanced together: 16 grayscale streams
# at each of 160x120, 320x240, 640x480 and 1280x720, ranks drawn from
# {5, 10, 15}, 3-10 % foreground as moving rectangles, noise 0.01.
BATCH_SIZES = ((160, 120), (320, 240), (640, 480), (1280, 720))


def batched_workload(seed: int = 4000, per_size: int = 16, n_frames: int = 500, sizes=BATCH_SIZES,
                     ranks=(5, 10, 15)):
    """[(SyntheticVideo, pROST parameter dict)] of the multi-stream workload."""
    rng = np.random.default_rng(seed)
    out = []
    sid = 0
    for (w, h) in sizes:
        for _ in range(per_size):
            k = int(rng.choice(ranks))
            fg = float(rng.uniform(0.03, 0.10))
            vid = SyntheticVideo(width=w, height=h, channels=1, k=k, n_frames=n_frames, fg_fraction=fg,
                                 shape="rect", n_shapes=3, jitter=0, seed=seed + 1 + sid, dtype="u8")
            prm = _params(vid.m, k, "u8")
            prm.update(width=w, height=h, channels=1, frame_dtype="u8")
            out.append((vid, prm))
            sid += 1
    return out


def window_workload(width: int = 320, height: int = 240, n: int = 64, k: int = 10, outliers: float = 0.05,
                    seed: int = 3000):
    """A window of n grayscale frames: a planted rank-k part U0 Y0 (U0
    orthonormal, the entries of Y0 N(0, 1) scaled to an entry deviation of
    0.1) with a fraction `outliers` of the entries replaced by U(0, 1).
    Returns (X n x m float32, U0 m x k, Y0 k x n, outlier mask n x m)."""
    rng = np.random.default_rng(seed)
    m = width * height
    U0 = random_orthonormal(m, k, rng)
    Y0 = rng.standard_normal((k, n)) * 0.1 * np.sqrt(m / k)
    X = (U0 @ Y0).T
    out = rng.random((n, m)) < outliers
    X[out] = rng.random(int(out.sum()))
    return np.ascontiguousarray(X, dtype=np.float32), U0, Y0, out
