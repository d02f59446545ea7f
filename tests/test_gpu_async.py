"""Pipelined host frames (prost_step_async / prost_wait) against the
synchronous host path, through the C ABI: the same frames give bit-identical
labels, backgrounds, subspaces and coefficients, statuses arrive in order,
a non-finite frame is reported by prost_wait and leaves the state untouched,
and the limits of the pipeline are enforced."""

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


@pytest.mark.parametrize("workload,k", [("gray160x120_k5", None), ("rgb640x480_k10", None),
                                        ("rgb640x480_k10", 15)])
def test_pipelined_frames_match_the_synchronous_path(workload, k):
    over = {} if k is None else {"k": k}
    vid, wp = synth.make_workload(workload, n_frames=9, **over)
    host = [np.ascontiguousarray(vid.frame(t)[0]) for t in range(9)]
    pinned = [torch.from_numpy(f).pin_memory() for f in host]
    a = pg.prost_init(gpu_params(wp, seed=4))
    b = pg.prost_init(gpu_params(wp, seed=4))
    try:
        ref_m, ref_bg = [], []
        for t in range(9):
            m_ = np.empty(vid.P, np.uint8)
            bg = np.empty(vid.m, np.float32)
            assert pg.prost_step(a, host[t], m_, bg) == pg.PROST_OK
            ref_m.append(m_)
            ref_bg.append(bg)
        outs = [(torch.empty(vid.P, dtype=torch.uint8).pin_memory(),
                 torch.empty(vid.m, dtype=torch.float32).pin_memory()) for _ in range(9)]
        for t in range(9):
            pg.prost_step_async(b, pinned[t], outs[t][0], outs[t][1])
            if t >= 1:
                assert pg.prost_wait(b) == pg.PROST_OK
        assert pg.prost_wait(b) == pg.PROST_OK
        for t in range(9):
            assert np.array_equal(outs[t][0].numpy(), ref_m[t]), t
            assert np.array_equal(outs[t][1].numpy(), ref_bg[t]), t
        Ua, ya = _export(a, vid)
        Ub, yb = _export(b, vid)
        assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
        assert pg.prost_get_stats(b).frames == 9
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_pipelined_bad_frame_and_limits():
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=4)
    host = [np.ascontiguousarray(vid.frame(t)[0]) for t in range(4)]
    bad = host[2].copy()
    bad.reshape(-1)[17] = np.nan
    h = pg.prost_init(gpu_params(wp, seed=4))
    try:
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_wait(h)                      # nothing in flight
        assert ei.value.code == pg.PROST_EINVAL
        masks = [np.empty(vid.P, np.uint8) for _ in range(3)]
        pg.prost_step_async(h, host[0], masks[0])
        pg.prost_step_async(h, host[1], masks[1])
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_step_async(h, host[2], masks[2])  # a third frame in flight
        assert ei.value.code == pg.PROST_EINVAL
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_step(h, host[2], masks[2])        # the synchronous path meanwhile
        assert ei.value.code == pg.PROST_EINVAL
        assert pg.prost_wait(h) == pg.PROST_OK
        assert pg.prost_wait(h) == pg.PROST_OK
        U0, y0 = _export(h, vid)
        pg.prost_step_async(h, bad, masks[2])
        assert pg.prost_wait(h) == pg.PROST_EBADFRAME
        assert pg.prost_sync(h) == pg.PROST_EBADFRAME
        U1, y1 = _export(h, vid)
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
        pg.prost_step_async(h, host[3], masks[2])
        assert pg.prost_wait(h) == pg.PROST_OK
        assert pg.prost_get_stats(h).frames == 3
    finally:
        pg.prost_destroy(h)
