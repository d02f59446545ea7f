"""Failure detection on the GPU without a GPU fault: the grid barrier is left
(by a host-side injection) the way a frame launch that gave up part-way
leaves it.  The next frame launch must detect it, refuse the frame without
touching the tracker's state, and prost_sync must report PROST_ETIMEOUT.
The tracker must then recover: the same frames give bit for bit what they
give on a tracker that never saw the fault.  No wait runs out here: a stale
barrier is caught when the launch starts.  This module sorts last, so no
other test depends on its outcome."""

import numpy as np
import pytest

import synth
import paper_1302_2073_gb300 as pg
from parity import gpu_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _export(h, vid):
    U = np.empty((vid.m, vid.k), np.float32)
    y = np.empty(vid.k)
    pg.prost_get_subspace(h, U, y)
    return U, y


@pytest.mark.parametrize("delta", [1 << 40, -1])
def test_stale_barrier_is_refused_reported_and_recovered(delta):
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=4)
    frames = [torch.from_numpy(vid.frame(t)[0]).cuda() for t in range(4)]
    mask = torch.empty(vid.P, dtype=torch.uint8, device="cuda")
    a = pg.prost_init(gpu_params(wp, seed=3))
    b = pg.prost_init(gpu_params(wp, seed=3))
    try:
        for h in (a, b):
            for t in range(2):
                pg.prost_step(h, frames[t], mask)
            assert pg.prost_sync(h) == pg.PROST_OK
        U0, y0 = _export(a, vid)
        frames_before = pg.prost_get_stats(a).frames

        pg.prost_inject_barrier_skew(a, delta)
        pg.prost_step(a, frames[2], mask)        # enqueued; the launch finds the barrier stale
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_sync(a)
        assert ei.value.code == pg.PROST_ETIMEOUT
        U1, y1 = _export(a, vid)
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
        assert pg.prost_get_stats(a).frames == frames_before

        for t in (2, 3):
            pg.prost_step(a, frames[t], mask)
            pg.prost_step(b, frames[t], mask)
        assert pg.prost_sync(a) == pg.PROST_OK
        assert pg.prost_sync(b) == pg.PROST_OK
        Ua, ya = _export(a, vid)
        Ub, yb = _export(b, vid)
        assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
        assert pg.prost_get_stats(a).frames == pg.prost_get_stats(b).frames == 4
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)
