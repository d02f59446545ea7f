"""Pins of the pre/post-processing oracle (Section 3.4) against closed forms
and library routines."""

import numpy as np
import pytest

from oracle import prepost as pp


def test_area_weights_hand_computed_five_to_two():
    # s = 2.5: output 0 covers [0, 2.5), output 1 covers [2.5, 5)
    A = pp.area_weights(5, 2)
    np.testing.assert_allclose(A, [[0.4, 0.4, 0.2, 0.0, 0.0], [0.0, 0.0, 0.2, 0.4, 0.4]], atol=1e-15)


@pytest.mark.parametrize("n_in,n_out", [(640, 160), (480, 120), (7, 3), (100, 100), (3, 8)])
def test_area_weights_rows_are_averages(n_in, n_out):
    A = pp.area_weights(n_in, n_out)
    np.testing.assert_allclose(A.sum(axis=1), 1.0, atol=1e-12)
    assert (A >= 0).all()
    # every input pixel contributes its full area in total
    np.testing.assert_allclose(A.sum(axis=0) * n_in / n_out, 1.0, atol=1e-12)


def test_resample_integer_factor_is_the_block_mean():
    rng = np.random.default_rng(0)
    f = rng.integers(0, 256, size=(3, 48, 64)).astype(np.uint8)
    out = pp.resample_area(f, 16, 12)
    ref = f.astype(np.float64).reshape(3, 12, 4, 16, 4).mean(axis=(2, 4))
    np.testing.assert_allclose(out, ref, rtol=1e-13)


def test_resample_identity_and_mass():
    rng = np.random.default_rng(1)
    f = rng.random((2, 17, 23))
    np.testing.assert_allclose(pp.resample_area(f, 23, 17), f, rtol=1e-13)
    out = pp.resample_area(f, 10, 6)
    np.testing.assert_allclose(out.sum() * (17 / 6) * (23 / 10), f.sum(), rtol=1e-12)
    # a square frame to a non-square size: each axis takes its own operator
    g = rng.random((1, 12, 12))
    out = pp.resample_area(g, 4, 3)
    assert out.shape == (1, 3, 4)
    np.testing.assert_allclose(out, g.reshape(1, 3, 4, 4, 3).mean(axis=(2, 4)), rtol=1e-13)


@pytest.mark.parametrize("signed", [False, True])
def test_running_norm_matches_the_closed_forms_and_freezes(signed):
    # unsigned intensities, and signed float frames (a pre-subtracted input),
    # where a sum of magnitudes instead of values would show
    rng = np.random.default_rng(2)
    if signed:
        frames = rng.standard_normal((7, 2, 5, 6)) - 0.3
    else:
        frames = rng.integers(0, 256, size=(7, 2, 5, 6)).astype(np.float64)
    rn = pp.RunningNorm(frames.shape[1:], i_init=4)
    for t in range(4):
        out = rn.apply(frames[t])
        seen = frames[: t + 1]
        mean = seen.mean(axis=0)
        std = seen.std(ddof=1) if seen.size > 1 else 1.0
        np.testing.assert_allclose(rn.mean, mean, rtol=1e-13)
        assert rn.std() == pytest.approx(std, rel=1e-12)
        np.testing.assert_allclose(out, (frames[t] - mean) / std, rtol=1e-12)
    m4, s4 = rn.mean.copy(), rn.std()
    for t in range(4, 7):
        out = rn.apply(frames[t])
        np.testing.assert_array_equal(rn.mean, m4)
        assert rn.std() == s4
        np.testing.assert_allclose(out, (frames[t] - m4) / s4, rtol=1e-13)


def test_running_norm_undefined_deviation_is_one():
    # one entry seen, or all entries equal: no sample deviation, divide by 1
    one = pp.RunningNorm((1, 1, 1), i_init=3)
    np.testing.assert_allclose(one.apply(np.full((1, 1, 1), 7.0)), 0.0)
    assert one.std() == 1.0
    assert one.apply(np.full((1, 1, 1), 9.0))[0, 0, 0] == pytest.approx((9.0 - 8.0) / np.sqrt(2.0), rel=1e-13)
    flat = pp.RunningNorm((2, 3, 4), i_init=2)
    out = flat.apply(np.full((2, 3, 4), 5.0))
    assert flat.std() == 1.0
    np.testing.assert_array_equal(out, 0.0)


def test_median_against_scipy_and_hand_cases():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    for p in (0.1, 0.5, 0.8):
        m = (rng.random((23, 31)) < p).astype(np.uint8)
        np.testing.assert_array_equal(pp.median3x3_mask(m), ndi.median_filter(m, size=3, mode="nearest"))
    iso = np.zeros((5, 5), np.uint8)
    iso[2, 2] = 1
    assert pp.median3x3_mask(iso).sum() == 0          # isolated pixel removed
    hole = np.ones((5, 5), np.uint8)
    hole[2, 2] = 0
    assert pp.median3x3_mask(hole).all()              # single-pixel hole filled
    corner = np.zeros((4, 4), np.uint8)
    corner[0, 0] = corner[0, 1] = corner[1, 0] = 1    # replicated border: 6 of 9 at (0, 0)
    assert pp.median3x3_mask(corner)[0, 0] == 1
