"""Many streams per tick (prost_batch) through the C ABI: per-stream parity
with the FP64 oracle for streams of mixed k, channels and frame types in one
tick, graph and direct launches bit-identical, the autotuner leaving the
trackers untouched, the kernel groups in turn or concurrent, a long run
across the rebase, and argument checks."""

import numpy as np
import pytest

import oracle
import synth
import paper_1302_2073_gb300 as pg
from parity import COST_RTOL, MASK_BAND, U_RTOL, Y_RTOL, gpu_params, matched_start, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _streams():
    """Six streams, three kernel families and two frame types; planes are
    16-byte multiples, as the batch requires."""
    spec = [(40, 32, 1, 5, "u8"), (64, 48, 3, 5, "u8"), (48, 32, 1, 12, "f32"),
            (80, 48, 3, 12, "u8"), (32, 32, 1, 3, "u8"), (96, 64, 1, 5, "u8")]
    out = []
    for i, (w, h, c, k, dt) in enumerate(spec):
        vid = synth.SyntheticVideo(w, h, c, k, n_frames=6, fg_fraction=0.06, seed=500 + i, dtype=dt)
        wp = synth.video._params(vid.m, k, dt)
        wp.update(width=w, height=h, channels=c, frame_dtype=dt)
        out.append((vid, wp))
    return out


def _export(h, vid):
    U = np.empty((vid.m, vid.k), np.float32)
    y = np.empty(vid.k)
    pg.prost_get_subspace(h, U, y)
    return U, y


@pytest.mark.parametrize("concurrent", [False, True])
def test_one_tick_matches_the_oracle_for_every_stream(concurrent):
    streams = _streams()
    b = pg.prost_batch_init([gpu_params(wp) for _, wp in streams])
    try:
        pg.prost_batch_set_concurrent(b, concurrent)
        assert pg.prost_batch_get_concurrent(b) == concurrent
        starts, frames, masks = [], [], []
        for i, (vid, wp) in enumerate(streams):
            st = oracle.initial_state(synth.random_orthonormal(vid.m, vid.k, 30 + i), vid.P)
            prm_o = oracle_params(wp)
            for t in range(2):
                oracle.frame_step(prm_o, st, vid.frame(t)[0])
            U32, U64, y64 = matched_start(st.U, st.y)
            h = pg.prost_batch_stream(b, i)
            pg.prost_set_subspace(h, U32, y64)
            pg.prost_set_labels(h, st.labels)
            pg.prost_set_frame_index(h, st.i)
            starts.append(oracle.OracleState(U64.copy(), y64.copy(), st.labels.copy(), st.i))
            frames.append(torch.from_numpy(vid.frame(2)[0]).cuda())
            masks.append(torch.empty(vid.P, dtype=torch.uint8, device="cuda"))
        pg.prost_batch_step(b, frames, masks)
        pg.prost_batch_sync(b)
        ctas, ngroups, alpha, graph = pg.prost_batch_plan(b, len(streams))
        assert ngroups == 4 and all(c >= 1 for c in ctas)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        if concurrent:  # every CTA of every group resident at once
            assert sum(ctas) <= sms
        for i, (vid, wp) in enumerate(streams):
            h = pg.prost_batch_stream(b, i)
            res = oracle.frame_step(oracle_params(wp), starts[i], vid.frame(2)[0])
            stats = pg.prost_get_stats(h)
            Ug, yg = _export(h, vid)
            n_cg = wp["n_cg"]
            cost = np.array(stats.cost[:n_cg + 1])
            np.testing.assert_allclose(cost, np.array(res.trace.cost[:n_cg + 1]), rtol=COST_RTOL)
            assert np.linalg.norm(yg - starts[i].y) <= Y_RTOL * np.linalg.norm(starts[i].y)
            assert np.linalg.norm(Ug - starts[i].U) <= U_RTOL * np.linalg.norm(starts[i].U)
            got = masks[i].cpu().numpy()
            r = np.abs(res.residual.reshape(vid.channels, vid.P)).max(axis=0)
            excused = np.abs(r - wp["delta"]) <= MASK_BAND
            assert ((got != res.labels) & ~excused).sum() == 0, f"stream {i}"
    finally:
        pg.prost_batch_destroy(b)


def _run(streams, graph, ticks, concurrent=False):
    b = pg.prost_batch_init([gpu_params(wp, seed=7) for _, wp in streams])
    try:
        pg.prost_batch_set_graph(b, graph)
        pg.prost_batch_set_concurrent(b, concurrent)
        fr = [[torch.from_numpy(v.frame(t % v.n_frames)[0]).cuda() for v, _ in streams] for t in range(ticks)]
        ms = [torch.empty(v.P, dtype=torch.uint8, device="cuda") for v, _ in streams]
        for t in range(ticks):
            pg.prost_batch_step(b, fr[t], ms)
        pg.prost_batch_sync(b)
        return [_export(pg.prost_batch_stream(b, i), v) for i, (v, _) in enumerate(streams)], \
            [m.cpu().numpy() for m in ms]
    finally:
        pg.prost_batch_destroy(b)


@pytest.mark.parametrize("concurrent", [False, True])
def test_graph_and_direct_launches_are_bit_identical(concurrent):
    streams = _streams()
    a, ma = _run(streams, True, 5, concurrent)
    d, md = _run(streams, False, 5, concurrent)
    for (Ua, ya), (Ud, yd) in zip(a, d):
        assert np.array_equal(Ua, Ud) and np.array_equal(ya, yd)
    for x, y in zip(ma, md):
        assert np.array_equal(x, y)


def test_concurrent_groups_track_the_serial_ones():
    # the CTA splits differ, so do the summation orders: the same subspaces to
    # FP32 rounding after five ticks
    streams = _streams()
    a, ma = _run(streams, True, 5, False)
    c, mc = _run(streams, True, 5, True)
    for (Ua, ya), (Uc, yc) in zip(a, c):
        assert np.linalg.norm(Ua - Uc) <= 1e-5 * np.linalg.norm(Ua)
        assert np.linalg.norm(ya - yc) <= 1e-5 * np.linalg.norm(ya)
    for x, y in zip(ma, mc):
        assert (x != y).mean() < 1e-3


def test_tuner_leaves_the_trackers_where_they_were():
    streams = _streams()
    b = pg.prost_batch_init([gpu_params(wp, seed=9) for _, wp in streams])
    try:
        fr = [torch.from_numpy(v.frame(0)[0]).cuda() for v, _ in streams]
        pg.prost_batch_step(b, fr)
        pg.prost_batch_sync(b)
        before = [_export(pg.prost_batch_stream(b, i), v) for i, (v, _) in enumerate(streams)]
        idx_before = [pg.prost_get_stats(pg.prost_batch_stream(b, i)).frames for i in range(len(streams))]
        ms = pg.prost_batch_tune(b, fr, ticks=3)
        after = [_export(pg.prost_batch_stream(b, i), v) for i, (v, _) in enumerate(streams)]
        idx_after = [pg.prost_get_stats(pg.prost_batch_stream(b, i)).frames for i in range(len(streams))]
        ctas, ngroups, alpha, graph = pg.prost_batch_plan(b, len(streams))
        # the tuned plan keeps working
        pg.prost_batch_step(b, fr)
        pg.prost_batch_sync(b)
    finally:
        pg.prost_batch_destroy(b)
    assert ms > 0 and alpha in (0.5, 0.75, 1.0)
    for (U0, y0), (U1, y1) in zip(before, after):
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
    assert idx_before == idx_after


def test_long_run_across_the_rebase():
    streams = [s for s in _streams() if s[0].m <= 4000][:3]
    b = pg.prost_batch_init([gpu_params(wp, seed=11) for _, wp in streams])
    try:
        fr = [[torch.from_numpy(v.frame(t)[0]).cuda() for v, _ in streams] for t in range(6)]
        for t in range(1100):
            pg.prost_batch_step(b, fr[t % 6])
        pg.prost_batch_sync(b)
        for i, (v, _) in enumerate(streams):
            U, _ = _export(pg.prost_batch_stream(b, i), v)
            np.testing.assert_allclose(U.T.astype(np.float64) @ U, np.eye(v.k), atol=2e-6)
            assert pg.prost_get_stats(pg.prost_batch_stream(b, i)).frames == 1100
    finally:
        pg.prost_batch_destroy(b)


def test_unaligned_frames_are_rejected():
    streams = _streams()[:2]
    b = pg.prost_batch_init([gpu_params(wp) for _, wp in streams])
    try:
        base = [torch.zeros(v.m + 16, dtype=torch.uint8, device="cuda") for v, _ in streams]
        with pytest.raises(pg.ProstError):
            pg.prost_batch_step(b, [x.data_ptr() + 1 for x in base])
    finally:
        pg.prost_batch_destroy(b)
