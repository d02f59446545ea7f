"""FP64 reference of pROST's pre- and post-processing (arXiv:1302.2073,
Section 3.4).  Test infrastructure only: tests, the smoke check and the
benchmark's CPU baseline use it; the product path never does.

Pre-processing (Section 3.4):
  * the frames are resampled to a fixed size (160 x 120 in the paper);
  * during the initialisation phase (the first i_init frames) the running
    average of the frames is maintained per entry and subtracted from every
    frame; after the phase it is kept fixed;
  * the intensities are divided by the sample standard deviation over all
    pixels of the initialisation phase (one number, running during the phase,
    fixed after it).
Post-processing (Section 3.4): a 3 x 3 median filter on the foreground mask.

Readings where the paper is silent:
  * resampling is area averaging: output pixel (i, j) is the mean of the input
    over its footprint [j W/w, (j+1) W/w) x [i H/h, (i+1) H/h), partially
    covered input pixels weighted by the covered fraction (exactly the block
    mean for integer factors); channels are resampled independently;
  * the running statistics include the current frame: frame t of the phase is
    normalised with the mean of frames 0..t and the deviation of all entries of
    frames 0..t (the deviation of a single entry is undefined, so frame 0 of a
    one-entry image uses 1);
  * the median filter replicates the border pixels; on a binary mask the
    median of 9 values is 1 exactly when at least 5 of them are 1.
"""

from __future__ import annotations

import numpy as np


def area_weights(n_in: int, n_out: int) -> np.ndarray:
    """n_out x n_in matrix A with A[i, q] = |[q, q+1) ∩ [i s, (i+1) s)| / s,
    s = n_in / n_out: the row-averaging operator of area resampling."""
    s = n_in / n_out
    A = np.zeros((n_out, n_in))
    for i in range(n_out):
        lo, hi = i * s, (i + 1) * s
        for q in range(int(np.floor(lo)), min(n_in, int(np.ceil(hi)))):
            ov = min(hi, q + 1) - max(lo, q)
            if ov > 0:
                A[i, q] = ov / s
    return A


def resample_area(frame: np.ndarray, w_out: int, h_out: int) -> np.ndarray:
    """frame: channels x H x W (any numeric type) -> channels x h_out x w_out (FP64)."""
    f = np.asarray(frame, dtype=np.float64)
    C, H, W = f.shape
    Ay = area_weights(H, h_out)
    Ax = area_weights(W, w_out)
    return np.stack([Ay @ f[c] @ Ax.T for c in range(C)])


class RunningNorm:
    """Running mean (per entry) and standard deviation (all entries) over the
    first i_init frames, then fixed (Section 3.4)."""

    def __init__(self, shape, i_init: int):
        self.i_init = i_init
        self.n = 0
        self.mean = np.zeros(shape)
        self.s1 = 0.0   # sum of all entries seen in the phase
        self.s2 = 0.0   # sum of their squares
        self.cnt = 0    # entries seen in the phase

    def std(self) -> float:
        if self.cnt < 2:
            return 1.0
        var = (self.s2 - self.s1 * self.s1 / self.cnt) / (self.cnt - 1)
        return float(np.sqrt(max(var, 0.0))) if var > 0 else 1.0

    def apply(self, v: np.ndarray) -> np.ndarray:
        """Normalise one frame (updating the statistics during the phase)."""
        v = np.asarray(v, dtype=np.float64)
        if self.n < self.i_init:
            self.n += 1
            self.mean += (v - self.mean) / self.n
            self.s1 += float(v.sum())
            self.s2 += float((v * v).sum())
            self.cnt += v.size
        return (v - self.mean) / self.std()


def median3x3_mask(mask: np.ndarray) -> np.ndarray:
    """3 x 3 median of a binary H x W mask, border pixels replicated: the
    majority (at least 5 of 9) of each neighbourhood."""
    m = (np.asarray(mask) != 0).astype(np.int64)
    H, W = m.shape
    p = np.pad(m, 1, mode="edge")
    count = np.zeros((H, W), dtype=np.int64)
    for dy in range(3):
        for dx in range(3):
            count += p[dy:dy + H, dx:dx + W]
    return (count >= 5).astype(np.uint8)
