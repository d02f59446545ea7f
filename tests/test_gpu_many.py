"""prost_step_many(): n frames of one stream per call.  In the resident form
they run in one launch whose CTAs keep their rows and labels in shared memory
from frame to frame; the results must be those of n prost_step() calls, bit
for bit (the same operations in the same order), through rejected frames, the
periodic rebase, host buffers and an aborted launch."""

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


def _export(h, m, k):
    U = np.empty((m, k), np.float32)
    y = np.empty(k)
    pg.prost_get_subspace(h, U, y)
    return U, y


def _stats_tuple(st):
    return (st.frames, st.bad_frames, st.n_foreground, tuple(st.cost), tuple(st.gnorm), st.pi_norm, st.theta,
            st.updated, st.pi_explicit)


def _pair(wp, **over):
    a = pg.prost_init(gpu_params(wp, form=pg.PROST_FORM_RESIDENT, seed=7, **over))
    b = pg.prost_init(gpu_params(wp, form=pg.PROST_FORM_RESIDENT, seed=7, **over))
    assert pg.prost_get_stats(a).form == pg.PROST_FORM_RESIDENT
    return a, b


def _compare(a, b, m, k):
    Ua, ya = _export(a, m, k)
    Ub, yb = _export(b, m, k)
    assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
    assert _stats_tuple(pg.prost_get_stats(a)) == _stats_tuple(pg.prost_get_stats(b))


@pytest.mark.parametrize("workload,over", [
    ("rgb640x480_k10", {}),                                   # about 86 % of the rows resident
    ("rgb640x480_k10", {"width": 160, "height": 120}),        # all rows resident
    ("rgb640x480_k10", {"width": 160, "height": 120, "u_dtype": "bf16"}),
    ("gray160x120_k5", {"width": 37, "height": 29}),          # ragged tail, odd P, float frames
])
def test_many_frames_equal_single_frames_bit_for_bit(workload, over):
    u_dtype = over.pop("u_dtype", "f32")
    vid, wp = synth.make_workload(workload, n_frames=6, **over)
    a, b = _pair(wp, u_dtype=u_dtype)
    try:
        frames = torch.from_numpy(vid.frames(0, 6)).cuda()
        ma = torch.empty((6, vid.P), dtype=torch.uint8, device="cuda")
        mb = torch.empty((6, vid.P), dtype=torch.uint8, device="cuda")
        assert pg.prost_step_many(a, frames, 6, ma) == pg.PROST_OK
        for t in range(6):
            pg.prost_step(b, frames[t], mb[t])
        assert pg.prost_sync(a) == pg.PROST_OK and pg.prost_sync(b) == pg.PROST_OK
        assert torch.equal(ma, mb)
        _compare(a, b, vid.m, vid.k)
        # and the next frames continue alike
        assert pg.prost_step_many(a, frames[:3], 3, ma[:3]) == pg.PROST_OK
        for t in range(3):
            pg.prost_step(b, frames[t], mb[t])
        assert torch.equal(ma[:3], mb[:3])
        _compare(a, b, vid.m, vid.k)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_host_buffers_and_a_rejected_frame_inside_the_launch():
    vid, wp = synth.make_workload("gray160x120_k5", width=64, height=48, n_frames=5)
    a, b = _pair(wp)
    try:
        host = np.ascontiguousarray(vid.frames(0, 5))
        host[2].reshape(-1)[17] = np.nan  # frame 2 is rejected, the others run
        ma = np.full((5, vid.P), 7, np.uint8)
        assert pg.prost_step_many(a, host, 5, ma) == pg.PROST_OK  # the last frame's status
        assert pg.prost_sync(a) == pg.PROST_EBADFRAME  # sticky until this call
        mb = np.empty((5, vid.P), np.uint8)
        for t in range(5):
            rc = pg.prost_step(b, host[t], mb[t])
            assert rc == (pg.PROST_EBADFRAME if t == 2 else pg.PROST_OK)
        assert pg.prost_sync(b) == pg.PROST_EBADFRAME
        for t in (0, 1, 3, 4):
            assert np.array_equal(ma[t], mb[t])
        _compare(a, b, vid.m, vid.k)
        assert pg.prost_get_stats(a).bad_frames == 1
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_a_call_across_the_stored_basis_rebase():
    # the stored rows are rebased every 1,024 frames: a call across that point
    # runs as two launches with the rebase between them
    vid = synth.SyntheticVideo(32, 24, 1, 3, n_frames=40, fg_fraction=0.05, walk_sigma=0.2, seed=41, dtype="f32")
    wp = synth.video._params(vid.m, vid.k, "f32")
    wp.update(width=32, height=24, channels=1, frame_dtype="f32")
    a, b = _pair(wp)
    try:
        frames = torch.from_numpy(vid.frames(0, 40)).cuda()
        m = torch.empty(vid.P, dtype=torch.uint8, device="cuda")
        for t in range(1000):
            pg.prost_step(a, frames[t % 40], m)
            pg.prost_step(b, frames[t % 40], m)
        ma = torch.empty((40, vid.P), dtype=torch.uint8, device="cuda")
        mb = torch.empty((40, vid.P), dtype=torch.uint8, device="cuda")
        assert pg.prost_step_many(a, frames, 40, ma) == pg.PROST_OK
        for t in range(40):
            pg.prost_step(b, frames[t], mb[t])
        assert pg.prost_sync(a) == pg.PROST_OK and pg.prost_sync(b) == pg.PROST_OK
        assert torch.equal(ma, mb)
        _compare(a, b, vid.m, vid.k)
        assert pg.prost_get_stats(a).frames == 1040
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_an_aborted_launch_leaves_the_state_and_recovers():
    vid, wp = synth.make_workload("gray160x120_k5", width=64, height=48, n_frames=4)
    a, b = _pair(wp)
    try:
        frames = torch.from_numpy(vid.frames(0, 4)).cuda()
        m = torch.empty((4, vid.P), dtype=torch.uint8, device="cuda")
        pg.prost_step_many(a, frames, 2, m)
        pg.prost_step_many(b, frames, 2, m)
        assert pg.prost_sync(a) == pg.PROST_OK and pg.prost_sync(b) == pg.PROST_OK
        U0, y0 = _export(a, vid.m, vid.k)
        pg.prost_inject_wait_timeout(a, 2, 20000)  # the first frame's third barrier gives up
        pg.prost_step_many(a, frames, 4, m)
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_sync(a)
        assert ei.value.code == pg.PROST_ETIMEOUT
        U1, y1 = _export(a, vid.m, vid.k)
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
        pg.prost_step_many(a, frames, 4, m)
        pg.prost_step_many(b, frames, 4, m)
        assert pg.prost_sync(a) == pg.PROST_OK and pg.prost_sync(b) == pg.PROST_OK
        _compare(a, b, vid.m, vid.k)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_other_forms_run_one_launch_per_frame():
    vid, wp = synth.make_workload("gray160x120_k5", width=64, height=48, n_frames=3)
    a = pg.prost_init(gpu_params(wp, form=pg.PROST_FORM_GRID, seed=7))
    b = pg.prost_init(gpu_params(wp, form=pg.PROST_FORM_GRID, seed=7))
    try:
        frames = torch.from_numpy(vid.frames(0, 3)).cuda()
        ma = torch.empty((3, vid.P), dtype=torch.uint8, device="cuda")
        mb = torch.empty((3, vid.P), dtype=torch.uint8, device="cuda")
        pg.prost_step_many(a, frames, 3, ma)
        for t in range(3):
            pg.prost_step(b, frames[t], mb[t])
        assert pg.prost_sync(a) == pg.PROST_OK and pg.prost_sync(b) == pg.PROST_OK
        assert torch.equal(ma, mb)
        _compare(a, b, vid.m, vid.k)
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_step_many(a, frames, 0, ma)
        assert ei.value.code == pg.PROST_EINVAL
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


@pytest.mark.parametrize("form", [pg.PROST_FORM_RESIDENT, pg.PROST_FORM_GRID])
def test_pipelined_many_frame_calls_equal_the_synchronous_calls(form):
    """prost_step_many_async with page-locked host frames, two calls in flight
    and growing call sizes, against prost_step_many on the same frames: masks,
    subspace, coefficients and statistics bit for bit, statuses in order."""
    vid, wp = synth.make_workload("rgb640x480_k10", width=160, height=120, n_frames=14)
    a = pg.prost_init(gpu_params(wp, form=form, seed=7))
    b = pg.prost_init(gpu_params(wp, form=form, seed=7))
    try:
        host = torch.from_numpy(np.ascontiguousarray(vid.frames(0, 14))).pin_memory()
        sizes = [2, 4, 4, 3, 1]  # 14 frames; the slots grow from 2 to 4
        outs, starts = [], []
        f0 = 0
        for i, n in enumerate(sizes):
            mo = torch.empty((n, vid.P), dtype=torch.uint8).pin_memory()
            outs.append(mo)
            starts.append(f0)
            assert pg.prost_step_many_async(a, host[f0:f0 + n], n, mo) == pg.PROST_OK
            if i >= 1:
                assert pg.prost_wait(a) == pg.PROST_OK
            f0 += n
        assert pg.prost_wait(a) == pg.PROST_OK
        with pytest.raises(pg.ProstError):
            pg.prost_wait(a)
        ref = np.empty((14, vid.P), np.uint8)
        f0 = 0
        for n in sizes:
            assert pg.prost_step_many(b, host[f0:f0 + n].numpy(), n, ref[f0:f0 + n]) == pg.PROST_OK
            f0 += n
        for mo, s0, n in zip(outs, starts, sizes):
            assert np.array_equal(mo.numpy(), ref[s0:s0 + n])
        assert pg.prost_sync(a) == pg.PROST_OK and pg.prost_sync(b) == pg.PROST_OK
        _compare(a, b, vid.m, vid.k)
        # a third call while two are in flight is refused
        m1 = torch.empty((2, vid.P), dtype=torch.uint8).pin_memory()
        pg.prost_step_many_async(a, host[:2], 2, m1)
        pg.prost_step_many_async(a, host[2:4], 2, m1)
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_step_many_async(a, host[4:6], 2, m1)
        assert ei.value.code == pg.PROST_EINVAL
        assert pg.prost_wait(a) == pg.PROST_OK and pg.prost_wait(a) == pg.PROST_OK
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)
