"""Life cycle of a tracker on the GPU: initial subspace, subspace import and
export, checkpoint and bit-identical resume, determinism, rejected frames,
rank-deficient subspaces, host and device buffers."""

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


def _wp(**over):
    vid, wp = synth.make_workload("rgb640x480_k10", width=48, height=36, n_frames=12)
    wp = dict(wp, **over)
    return vid, wp


def _subspace(h, m, k):
    U = np.empty((m, k), dtype=np.float32)
    y = np.empty(k)
    pg.prost_get_subspace(h, U, y)
    return U, y


def test_initial_subspace_is_orthonormal_and_seeded():
    vid, wp = _wp()
    hs = [pg.prost_init(gpu_params(wp, seed=s)) for s in (1, 1, 2)]
    try:
        Us = [_subspace(h, vid.m, vid.k) for h in hs]
        for U, y in Us:
            np.testing.assert_allclose(U.T.astype(np.float64) @ U, np.eye(vid.k), atol=2e-6)
            assert np.all(y == 0)
        assert np.array_equal(Us[0][0], Us[1][0])
        assert not np.allclose(Us[0][0], Us[2][0])
    finally:
        for h in hs:
            pg.prost_destroy(h)


def test_subspace_roundtrip():
    vid, wp = _wp()
    U0 = synth.random_orthonormal(vid.m, vid.k, 5).astype(np.float32)
    y0 = np.arange(1.0, vid.k + 1)
    h = pg.prost_init(gpu_params(wp))
    try:
        pg.prost_set_subspace(h, U0, y0)
        U, y = _subspace(h, vid.m, vid.k)
        np.testing.assert_allclose(U, U0, atol=1e-6)
        np.testing.assert_allclose(U.astype(np.float64) @ y, U0.astype(np.float64) @ y0, atol=1e-5)
        # device buffers give the same
        Ud = torch.empty((vid.m, vid.k), dtype=torch.float32, device="cuda")
        yd = torch.empty(vid.k, dtype=torch.float64, device="cuda")
        pg.prost_get_subspace(h, Ud, yd)
        torch.cuda.synchronize()
        assert np.array_equal(Ud.cpu().numpy(), U) and np.array_equal(yd.cpu().numpy(), y)
    finally:
        pg.prost_destroy(h)


def test_rank_deficient_subspace_is_rejected():
    vid, wp = _wp()
    U0 = synth.random_orthonormal(vid.m, vid.k, 5).astype(np.float32)
    U0[:, 3] = 0.0
    h = pg.prost_init(gpu_params(wp))
    try:
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_set_subspace(h, U0)
        assert ei.value.code == pg.PROST_ENOTSPD
    finally:
        pg.prost_destroy(h)


def _run(h, vid, t0, n, device=True):
    masks = []
    for t in range(t0, t0 + n):
        f, _ = vid.frame(t)
        if device:
            fd = torch.from_numpy(f).cuda()
            md = torch.empty(vid.P, dtype=torch.uint8, device="cuda")
            pg.prost_step(h, fd, md)
            masks.append(md)
        else:
            m = np.empty(vid.P, dtype=np.uint8)
            assert pg.prost_step(h, f, m) == pg.PROST_OK
            masks.append(m)
    if device:
        assert pg.prost_sync(h) == pg.PROST_OK
        masks = [m.cpu().numpy() for m in masks]
    return np.stack(masks), _subspace(h, vid.m, vid.k)


def test_runs_are_deterministic_and_host_equals_device():
    vid, wp = _wp()
    a, b = pg.prost_init(gpu_params(wp, seed=3)), pg.prost_init(gpu_params(wp, seed=3))
    try:
        ma, (Ua, ya) = _run(a, vid, 0, 8, device=True)
        mb, (Ub, yb) = _run(b, vid, 0, 8, device=False)
        assert np.array_equal(ma, mb) and np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_checkpoint_resume_is_bit_identical():
    vid, wp = _wp()
    a = pg.prost_init(gpu_params(wp, seed=4))
    b = pg.prost_init(gpu_params(wp, seed=99))
    try:
        _run(a, vid, 0, 4)
        state = pg.prost_get_state(a)
        ma, (Ua, ya) = _run(a, vid, 4, 5)
        pg.prost_set_state(b, state)
        mb, (Ub, yb) = _run(b, vid, 4, 5)
        assert np.array_equal(ma, mb) and np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
        assert pg.prost_get_stats(a).frames == pg.prost_get_stats(b).frames == 9
        # a state of another geometry is refused
        vid2, wp2 = _wp(width=40)
        c = pg.prost_init(gpu_params(wp2))
        try:
            with pytest.raises(pg.ProstError):
                pg.prost_set_state(c, state)
            with pytest.raises(pg.ProstError):
                pg.prost_set_state(c, state[:100])
        finally:
            pg.prost_destroy(c)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_non_finite_frame_is_skipped_and_state_kept():
    vid = synth.SyntheticVideo(40, 30, 1, 4, n_frames=5, seed=8, dtype="f32")
    wp = synth.video._params(vid.m, vid.k, "f32")
    wp.update(width=40, height=30, channels=1, frame_dtype="f32")
    h = pg.prost_init(gpu_params(wp))
    try:
        _run(h, vid, 0, 2, device=False)
        U0, y0 = _subspace(h, vid.m, vid.k)
        st0 = bytes(pg.prost_get_state(h))
        f, _ = vid.frame(2)
        bad = f.copy()
        bad.flat[123] = np.nan
        m = np.empty(vid.P, dtype=np.uint8)
        assert pg.prost_step(h, bad, m) == pg.PROST_EBADFRAME
        bad.flat[123] = np.inf
        fd = torch.from_numpy(bad).cuda()
        pg.prost_step(h, fd, torch.empty(vid.P, dtype=torch.uint8, device="cuda"))
        assert pg.prost_sync(h) == pg.PROST_EBADFRAME
        assert pg.prost_sync(h) == pg.PROST_OK  # flags cleared
        U1, y1 = _subspace(h, vid.m, vid.k)
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
        st = pg.prost_get_stats(h)
        assert st.frames == 2 and st.bad_frames == 2 and st.status == pg.PROST_EBADFRAME
        # the next good frame proceeds as if the bad ones never came
        assert pg.prost_step(h, f, m) == pg.PROST_OK
        ref = pg.prost_init(gpu_params(wp))
        try:
            pg.prost_set_state(ref, st0)
            m2 = np.empty(vid.P, dtype=np.uint8)
            assert pg.prost_step(ref, f, m2) == pg.PROST_OK
            assert np.array_equal(m, m2)
            assert np.array_equal(_subspace(h, vid.m, vid.k)[0], _subspace(ref, vid.m, vid.k)[0])
        finally:
            pg.prost_destroy(ref)
    finally:
        pg.prost_destroy(h)


def test_stream_ordering_on_a_caller_stream():
    vid, wp = _wp()
    s = torch.cuda.Stream()
    h = pg.prost_init(gpu_params(wp, seed=6), stream=s)
    ref = pg.prost_init(gpu_params(wp, seed=6))
    try:
        with torch.cuda.stream(s):
            fr = [torch.from_numpy(vid.frame(t)[0]).cuda() for t in range(5)]
            outs = [torch.empty(vid.P, dtype=torch.uint8, device="cuda") for _ in range(5)]
        for f, o in zip(fr, outs):
            pg.prost_step(h, f, o)
        assert pg.prost_sync(h) == pg.PROST_OK
        mr, _ = _run(ref, vid, 0, 5, device=False)
        assert np.array_equal(np.stack([o.cpu().numpy() for o in outs]), mr)
    finally:
        pg.prost_destroy(h)
        pg.prost_destroy(ref)
