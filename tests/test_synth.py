"""The seeded synthetic video: determinism and the stated recipe."""

import numpy as np
import pytest

import synth


def test_frames_are_deterministic_and_random_access():
    v1, _ = synth.make_workload("gray160x120_k5")
    v2, _ = synth.make_workload("gray160x120_k5")
    f7a, g7a = v1.frame(7)
    _ = v2.frame(3)
    f7b, g7b = v2.frame(7)
    assert np.array_equal(f7a, f7b) and np.array_equal(g7a, g7b)
    assert f7a.dtype == np.float32 and f7a.shape == (1, 120, 160)


def test_recipe_statistics():
    vid, prm = synth.make_workload("rgb640x480_k10", n_frames=4)
    f, gt = vid.frame(2)
    assert f.dtype == np.uint8 and f.shape == (3, 480, 640)
    assert f.flags.c_contiguous and gt.flags.c_contiguous
    frac = gt.mean()
    assert 0.05 < frac < 0.09  # ~8% foreground (overlaps may lower it)
    b = vid.background(2) - vid.offset
    assert 0.08 < b.std() < 0.12  # per-entry background std close to the amplitude
    np.testing.assert_allclose(vid.U0.T @ vid.U0, np.eye(10), atol=1e-12)
    assert prm["in_scale"] == 1 / 255 and prm["in_offset"] == 0.5


def test_jitter_shifts_whole_frame_with_edge_replication():
    vid = synth.SyntheticVideo(32, 24, 1, 2, n_frames=3, fg_fraction=0.0, jitter=2,
                               noise_sigma=0.0, seed=5, dtype="f32")
    f, _ = vid.frame(1)
    b = vid.background(1).astype(np.float32)
    # some integer shift in [-2, 2]^2 with clamped indices reproduces the frame
    hits = 0
    for dx in range(-2, 3):
        for dy in range(-2, 3):
            rows = np.clip(np.arange(24) - dy, 0, 23)
            cols = np.clip(np.arange(32) - dx, 0, 31)
            if np.allclose(np.clip(b[:, rows][:, :, cols], 0, 1), f, atol=1e-6):
                hits += 1
    assert hits >= 1


def test_device_video_follows_the_host_recipe():
    """The torch generator (run here on the CPU) shares the host stream's
    planted subspace, walk and shapes: its noiseless pieces match the numpy
    ones, its frames are reproducible, and its draws stay in range."""
    torch = pytest.importorskip("torch")
    from synth.video_gpu import DeviceVideo
    vid, _ = synth.make_workload("rgb640x480_k10", width=64, height=48, n_frames=5)
    dv = DeviceVideo(vid, "cpu")
    for t in (0, 3):
        assert np.array_equal(dv.shape_mask(t).numpy(), vid.shape_mask(t))
        b = (vid.offset + vid.scale * (dv.U0 @ dv.Y0[t])).numpy().reshape(vid.channels, vid.height, vid.width)
        np.testing.assert_allclose(b, vid.background(t), atol=1e-5)
        f1, f2 = dv.frame(t), dv.frame(t)
        assert f1.dtype == torch.uint8 and tuple(f1.shape) == (vid.channels, vid.height, vid.width)
        assert torch.equal(f1, f2)
    assert not torch.equal(dv.frame(0), dv.frame(1))
