"""Failure detection on the GPU without a GPU fault.

Two host-side injections stand in for a stalled or aborted frame:
* prost_inject_barrier_skew leaves the grid barrier the way a launch that gave
  up part-way leaves it; the next launch must refuse the frame at its start;
* prost_inject_wait_timeout makes one barrier of the next launch wait for an
  arrival that never comes, with a short spin limit, so the bounded wait itself
  runs out mid-frame (the window U-step has the same hook).
In each case the state must stay untouched, the error must be reported (by
prost_sync, and by prost_step itself on the host path, with its outputs left
unwritten), and the tracker must then give bit for bit what a tracker that
never saw the fault gives, also across the periodic rebase of the stored rows.
Nothing here faults or hangs the GPU: every wait is bounded and returns an
error status."""

import numpy as np
import pytest

import synth
import paper_1302_2073_gb300 as pg
from parity import gpu_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STALL_CYCLES = 200_000  # about 0.1 ms of SM clock: far below the default 2e9


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _export(h, vid):
    U = np.empty((vid.m, vid.k), np.float32)
    y = np.empty(vid.k)
    pg.prost_get_subspace(h, U, y)
    return U, y


def _grid_size(h):
    """The frame kernel's grid size: the smallest forward skew a launch can
    detect (smaller ones are refused by the injector itself)."""
    for d in range(1, 4096):
        try:
            pg.prost_inject_barrier_skew(h, d)
        except pg.ProstError as e:
            assert e.code == pg.PROST_EINVAL
            continue
        pg.prost_inject_barrier_skew(h, -d)  # put the count back
        return d
    raise AssertionError("no detectable skew found")


def _pair(wp, frames, n_before, form=pg.PROST_FORM_GRID):
    # the grid or resident form: the cluster form has no software barrier to disturb
    a = pg.prost_init(gpu_params(wp, seed=3, form=form))
    b = pg.prost_init(gpu_params(wp, seed=3, form=form))
    mask = torch.empty(frames[0].numel() // wp["channels"], dtype=torch.uint8, device="cuda")
    for h in (a, b):
        for t in range(n_before):
            pg.prost_step(h, frames[t % len(frames)], mask)
        assert pg.prost_sync(h) == pg.PROST_OK
    return a, b, mask


def _continue_and_compare(a, b, vid, frames, start, n, mask):
    for t in range(start, start + n):
        pg.prost_step(a, frames[t % len(frames)], mask)
        pg.prost_step(b, frames[t % len(frames)], mask)
    assert pg.prost_sync(a) == pg.PROST_OK
    assert pg.prost_sync(b) == pg.PROST_OK
    Ua, ya = _export(a, vid)
    Ub, yb = _export(b, vid)
    assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
    assert pg.prost_get_stats(a).frames == pg.prost_get_stats(b).frames


def _inject(kind, h):
    if kind == "skew_forward":
        pg.prost_inject_barrier_skew(h, 1 << 40)
    elif kind == "skew_backward":
        pg.prost_inject_barrier_skew(h, -1)
    elif kind == "skew_grid":
        pg.prost_inject_barrier_skew(h, _grid_size(h))
    elif kind.startswith("stall"):
        pg.prost_inject_wait_timeout(h, int(kind[5:]), STALL_CYCLES)
    else:
        raise ValueError(kind)


@pytest.mark.parametrize("form", [pg.PROST_FORM_GRID, pg.PROST_FORM_RESIDENT])
@pytest.mark.parametrize("kind", ["skew_forward", "skew_backward", "skew_grid", "stall0", "stall2", "stall5"])
def test_fault_is_refused_reported_and_recovered(kind, form):
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=4)
    frames = [torch.from_numpy(vid.frame(t)[0]).cuda() for t in range(4)]
    a, b, mask = _pair(wp, frames, 2, form)
    try:
        U0, y0 = _export(a, vid)
        frames_before = pg.prost_get_stats(a).frames
        _inject(kind, a)
        pg.prost_step(a, frames[2], mask)  # enqueued: refused at launch, or its wait runs out
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_sync(a)
        assert ei.value.code == pg.PROST_ETIMEOUT
        U1, y1 = _export(a, vid)
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
        assert pg.prost_get_stats(a).frames == frames_before
        _continue_and_compare(a, b, vid, frames, 2, 2, mask)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


@pytest.mark.parametrize("kind", ["skew_backward", "stall1"])
def test_host_frame_reports_the_fault_and_leaves_outputs_unwritten(kind):
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=4)
    host = [vid.frame(t)[0] for t in range(4)]
    frames = [torch.from_numpy(f).cuda() for f in host]
    a, b, mask = _pair(wp, frames, 2)
    try:
        _inject(kind, a)
        out = np.full(vid.P, 0xAB, np.uint8)
        bg = np.full(vid.m, -7.0, np.float32)
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_step(a, host[2], out, bg)
        assert ei.value.code == pg.PROST_ETIMEOUT
        assert np.all(out == 0xAB) and np.all(bg == -7.0)
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_sync(a)
        assert ei.value.code == pg.PROST_ETIMEOUT
        # the next host frame runs and writes its outputs
        assert pg.prost_step(a, host[2], out, bg) == pg.PROST_OK
        assert set(np.unique(out)) <= {0, 1}
        pg.prost_step(b, frames[2], mask)
        _continue_and_compare(a, b, vid, frames, 3, 1, mask)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


def test_the_cluster_form_takes_no_barrier_injection():
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=1)
    h = pg.prost_init(gpu_params(wp, seed=3, form=pg.PROST_FORM_CLUSTER))
    try:
        for inject in (lambda: pg.prost_inject_barrier_skew(h, -1),
                       lambda: pg.prost_inject_wait_timeout(h, 0, STALL_CYCLES)):
            with pytest.raises(pg.ProstError) as ei:
                inject()
            assert ei.value.code == pg.PROST_EINVAL
    finally:
        pg.prost_destroy(h)


def test_undetectable_forward_skew_is_rejected_by_the_injector():
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=1)
    h = pg.prost_init(gpu_params(wp, seed=3, form=pg.PROST_FORM_GRID))
    try:
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_inject_barrier_skew(h, 1)
        assert ei.value.code == pg.PROST_EINVAL
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_inject_wait_timeout(h, wp["n_cg"] + 1, STALL_CYCLES)
        assert ei.value.code == pg.PROST_EINVAL
    finally:
        pg.prost_destroy(h)


def test_recovery_keeps_the_rebase_on_its_frame():
    # the stored rows are rebased after every 1,024 completed frames; a frame
    # refused before that point must not move the rebase one frame earlier
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=8)
    frames = [torch.from_numpy(vid.frame(t)[0]).cuda() for t in range(8)]
    a, b, mask = _pair(wp, frames, 1020)
    try:
        pg.prost_inject_wait_timeout(a, 1, STALL_CYCLES)
        pg.prost_step(a, frames[4], mask)
        with pytest.raises(pg.ProstError):
            pg.prost_sync(a)
        _continue_and_compare(a, b, vid, frames, 1020, 10, mask)
        assert pg.prost_get_stats(a).frames == 1030
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)


@pytest.mark.parametrize("barrier", [1, 2])
def test_window_ustep_wait_runs_out(barrier):
    m, k, n = 320 * 240, 10, 8
    rng = np.random.default_rng(5)
    U = torch.from_numpy(synth.random_orthonormal(m, k, rng).astype(np.float32)).cuda()
    dU = torch.from_numpy((rng.standard_normal((m, k)) * 1e-3).astype(np.float32)).cuda()
    w = pg.prost_window_init(m, 1, k, n)
    try:
        ref = torch.empty_like(U)
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        pg.prost_window_ustep(w, U, dU, 0.5, ref, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        out = torch.full_like(U, -7.0)
        pg.prost_window_inject_wait_timeout(w, barrier, STALL_CYCLES)
        pg.prost_window_ustep(w, U, dU, 0.5, out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == -2
        assert bool((out == -7.0).all())
        pg.prost_window_ustep(w, U, dU, 0.5, out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out, ref)
    finally:
        pg.prost_window_destroy(w)
