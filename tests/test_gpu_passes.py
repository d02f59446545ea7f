"""The passes form (k chosen at run time, every k up to 32) against the FP64
oracle, through the C ABI: teacher-forced parity at k = 17..32, ragged uint8
planes, CG iteration counts, Step 2's degenerate points, a rejected frame, a
free run, a run across the stored-basis rebase with a checkpoint, the
benchmark frame size at k = 20 and 32, and reproducibility.  The same form at
k <= 16 is also run by the parametrised cases of test_gpu_parity.py and
test_gpu_degenerate.py."""

import numpy as np
import pytest

import oracle
import synth
import paper_1302_2073_gb300 as pg
from parity import PI_BAND, compare_step, gpu_params, gpu_step_from, matched_start, oracle_eta_norm, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _states(wp, vid, n, seed):
    prm_o = oracle_params(wp)
    st = oracle.initial_state(synth.random_orthonormal(vid.m, vid.k, seed), vid.P)
    out = []
    for t in range(n):
        out.append(st.copy())
        f, _ = vid.frame(t)
        oracle.frame_step(prm_o, st, f, want_residual=False)
    return out


def _teacher_forced(wp, vid, frames, seed=11, device=True, **gover):
    wpo = dict(wp, **gover)
    prm_o = oracle_params(wpo)
    states = _states(wpo, vid, max(frames) + 1, seed)
    h = pg.prost_init(gpu_params(wp, **gover))
    errs = []
    try:
        for t in frames:
            s = states[t]
            U32, U64, y64 = matched_start(s.U, s.y)
            f, _ = vid.frame(t)
            g = gpu_step_from(h, U32, s.y, s.labels, s.i, f, device=device, torch=torch)
            assert g.status == pg.PROST_OK
            assert g.stats.form == pg.PROST_FORM_PASSES
            e, _, _ = compare_step(prm_o, wpo, U64, y64, s.labels, s.i, f, g)
            errs.append(e)
    finally:
        pg.prost_destroy(h)
    return errs


@pytest.mark.parametrize("k", [17, 20, 24, 31, 32])
def test_subspace_dimensions_above_the_single_launch_forms(k):
    vid = synth.SyntheticVideo(50, 40, 1, k, n_frames=4, fg_fraction=0.05, seed=500 + k, dtype="f32")
    wp = synth.video._params(vid.m, k, "f32")
    wp.update(width=50, height=40, channels=1, frame_dtype="f32")
    print(_teacher_forced(wp, vid, [0, 2]))


@pytest.mark.parametrize("k", [20, 32])
def test_rgb_ragged_unaligned_planes_uint8(k):
    # P = 37*29 = 1073: planes off 4-byte boundaries, ragged tails in every tile
    vid = synth.SyntheticVideo(37, 29, 3, k, n_frames=6, fg_fraction=0.1, shape="ellipse",
                               jitter=1, seed=600 + k, dtype="u8")
    wp = synth.video._params(vid.m, k, "u8")
    wp.update(width=37, height=29, channels=3, frame_dtype="u8")
    _teacher_forced(wp, vid, [0, 1, 4])
    _teacher_forced(wp, vid, [1], device=False, mask_from=pg.PROST_MASK_PRE_UPDATE)


@pytest.mark.parametrize("n_cg", [0, 1, 12])
def test_cg_iteration_counts(n_cg):
    vid, wp = synth.make_workload("gray160x120_k5", width=40, height=30, k=20, n_frames=4)
    _teacher_forced(dict(wp, n_cg=n_cg), vid, [0, 2])


def test_cost_exponent_one():
    vid, wp = synth.make_workload("gray160x120_k5", width=40, height=30, k=18, n_frames=4)
    _teacher_forced(dict(wp, p=1.0, mu=1e-3), vid, [0, 2])


def _lsq(width, height, channels, k, **over):
    wp = dict(width=width, height=height, channels=channels, k=k, p=2.0, mu=0.01, delta=0.35,
              omega=1.0, t_init=0.5, t_min=1e-4, i_init=100, n_cg=0, in_scale=1.0, in_offset=0.5,
              frame_dtype="f32")
    wp.update(over)
    return wp


def _one_frame(wp, U32, U64, y, frame):
    P = wp["width"] * wp["height"]
    labels = np.zeros(P, np.uint8)
    y_raw = np.linalg.lstsq(U32.astype(np.float64), U64 @ y, rcond=None)[0]
    _, U64, y64 = matched_start(U32, y_raw)
    prm_o = oracle_params(wp)
    h = pg.prost_init(gpu_params(wp))
    try:
        g = gpu_step_from(h, U32, y_raw, labels, 0, frame, device=True, torch=torch)
        assert g.status == pg.PROST_OK and g.stats.form == pg.PROST_FORM_PASSES
    finally:
        pg.prost_destroy(h)
    err, _, res = compare_step(prm_o, wp, U64, y64, labels, 0, frame, g, pi_band=True)
    return g, err, res.trace, oracle_eta_norm(prm_o, U64, y64, labels, frame)


def test_degenerate_steps():
    k, W, H = 20, 64, 48
    m = W * H * 3
    rng = np.random.default_rng(71)
    U32, U64, _ = matched_start(synth.random_orthonormal(m, k, rng), np.zeros(k))
    wp = _lsq(W, H, 3, k)
    zero = (np.zeros(m) + wp["in_offset"]).astype(np.float32)
    # y = 0 on a zero frame: nothing to fit, Step 2 skipped
    g, err, tr, eta_n = _one_frame(dict(wp, n_cg=5), U32, U64, np.zeros(k), zero)
    assert tr.updated == 0 and g.stats.updated == 0 and g.stats.theta == 0.0
    assert np.all(g.y == 0.0) and not g.mask.any()
    # y != 0 on a zero frame: eta lies in span(U), the explicit pass forms |pi(eta)|
    g, err, tr, eta_n = _one_frame(wp, U32, U64, rng.standard_normal(k) * 3.0, zero)
    assert g.stats.pi_explicit == 1
    assert tr.pi_norm < 1e-12 * eta_n and g.stats.pi_norm < 1e-5 * eta_n


@pytest.mark.parametrize("ratio", [1e-3, 1e-2])
def test_eta_almost_in_span(ratio):
    k, W, H = 24, 96, 72
    m = W * H * 3
    rng = np.random.default_rng(80)
    U32, U64, _ = matched_start(synth.random_orthonormal(m, k, rng), np.zeros(k))
    y0 = rng.standard_normal(k) * 2.0
    d = rng.standard_normal(k)
    d *= 4.0 / np.linalg.norm(d)
    noise = rng.standard_normal(m) * (4.0 * ratio / np.sqrt(m))
    wp = _lsq(W, H, 3, k)
    frame = (U64 @ (y0 + d) + noise + wp["in_offset"]).astype(np.float32)
    g, err, tr, eta_n = _one_frame(wp, U32, U64, y0, frame)
    assert 0.3 * ratio < tr.pi_norm / eta_n < 3.0 * ratio
    assert tr.pi_norm > PI_BAND * eta_n
    assert g.stats.pi_explicit == 1 and g.stats.updated == 1 and tr.updated == 1
    assert err["theta"] <= 1e-4 and tr.theta > 1e-3


def test_rejected_frame_leaves_the_state():
    vid, wp = synth.make_workload("gray160x120_k5", width=48, height=40, k=20, n_frames=3)
    assert wp["frame_dtype"] == "f32"
    h = pg.prost_init(gpu_params(wp))
    try:
        f0 = vid.frame(0)[0]
        m = np.empty(vid.P, np.uint8)
        assert pg.prost_step(h, np.ascontiguousarray(f0, np.float32), m) == pg.PROST_OK
        U0 = np.empty((vid.m, vid.k), np.float32)
        y0 = np.empty(vid.k)
        pg.prost_get_subspace(h, U0, y0)
        before = pg.prost_get_stats(h)
        bad = np.array(f0, np.float32)
        bad.reshape(-1)[123] = np.nan
        m2 = np.full(vid.P, 7, np.uint8)
        assert pg.prost_step(h, bad, m2) == pg.PROST_EBADFRAME
        assert np.all(m2 == 7)  # outputs left unwritten
        U1 = np.empty_like(U0)
        y1 = np.empty_like(y0)
        pg.prost_get_subspace(h, U1, y1)
        after = pg.prost_get_stats(h)
        assert np.array_equal(U0, U1) and np.array_equal(y0, y1)
        assert after.frames == before.frames and after.bad_frames == before.bad_frames + 1
        assert pg.prost_sync(h) == pg.PROST_EBADFRAME
        assert pg.prost_step(h, np.ascontiguousarray(f0, np.float32), m) == pg.PROST_OK
    finally:
        pg.prost_destroy(h)


def _angle_max(A, B):
    qa, _ = np.linalg.qr(A.astype(np.float64))
    qb, _ = np.linalg.qr(B.astype(np.float64))
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def test_free_run_tracks_the_oracle():
    vid, wp = synth.make_workload("gray160x120_k5", k=20, n_frames=60)
    prm_o = oracle_params(wp)
    U32, U64, y64 = matched_start(synth.random_orthonormal(vid.m, vid.k, 9), np.zeros(vid.k))
    st = oracle.OracleState(U64.copy(), y64.copy(), np.zeros(vid.P, np.uint8), 0)
    h = pg.prost_init(gpu_params(wp))
    try:
        pg.prost_set_subspace(h, U32)
        dis, costs = [], []
        for t in range(60):
            f, _ = vid.frame(t)
            m = np.empty(vid.P, np.uint8)
            assert pg.prost_step(h, f, m) == pg.PROST_OK
            res = oracle.frame_step(prm_o, st, f, want_residual=False)
            dis.append(float((m != res.labels).mean()))
            costs.append(abs(pg.prost_get_stats(h).cost[0] - res.trace.cost[0]) / res.trace.cost[0])
        Ug = np.empty((vid.m, vid.k), np.float32)
        pg.prost_get_subspace(h, Ug, np.empty(vid.k))
    finally:
        pg.prost_destroy(h)
    ang = _angle_max(Ug, st.U)
    print("k = 20 free run: max angle", ang, "label disagreement", np.mean(dis), "cost", max(costs))
    assert ang < 1e-4
    assert np.mean(dis) < 1e-3 and max(dis) < 1e-2
    assert max(costs) < 1e-4


def test_run_across_the_rebase_resumes_from_a_checkpoint():
    vid = synth.SyntheticVideo(32, 24, 1, 17, n_frames=1100, fg_fraction=0.05, walk_sigma=0.2,
                               seed=37, dtype="f32")
    wp = synth.video._params(vid.m, vid.k, "f32")
    wp.update(width=32, height=24, channels=1, frame_dtype="f32", t_init=0.02, t_min=2e-3, i_init=50)
    prm_o = oracle_params(wp)
    U32, U64, y64 = matched_start(synth.random_orthonormal(vid.m, vid.k, 8), np.zeros(vid.k))
    st = oracle.OracleState(U64.copy(), y64.copy(), np.zeros(vid.P, np.uint8), 0)
    frames = vid.frames(0, 1100)
    a = pg.prost_init(gpu_params(wp))
    b = pg.prost_init(gpu_params(wp))
    try:
        pg.prost_set_subspace(a, U32)
        m = np.empty(vid.P, np.uint8)
        ck = None
        for t in range(1100):
            assert pg.prost_step(a, frames[t], m) == pg.PROST_OK
            oracle.frame_step(prm_o, st, frames[t], want_residual=False)
            if t == 1000:
                ck = pg.prost_get_state(a)
        Ua = np.empty((vid.m, vid.k), np.float32)
        ya = np.empty(vid.k)
        pg.prost_get_subspace(a, Ua, ya)
        pg.prost_set_state(b, ck)
        for t in range(1001, 1100):
            assert pg.prost_step(b, frames[t], m) == pg.PROST_OK
        Ub = np.empty_like(Ua)
        yb = np.empty_like(ya)
        pg.prost_get_subspace(b, Ub, yb)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)
    assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
    np.testing.assert_allclose(Ua.T.astype(np.float64) @ Ua, np.eye(vid.k), atol=2e-6)
    ang = _angle_max(Ua, st.U)
    print("k = 17, max angle after 1100 frames", ang)
    assert ang < 1e-3


@pytest.mark.parametrize("k", [20, 32])
def test_full_size_640x480_rgb(k):
    """The benchmark frame size (640x480 RGB, uint8 frames in device memory)
    at k = 20 and 32: teacher-forced parity of every output at frames 0, 1."""
    vid, wp = synth.make_workload("rgb640x480_k10", k=k, n_frames=2)
    print(_teacher_forced(wp, vid, [0, 1]))


def test_runs_are_reproducible_and_match_the_grid_form_at_k16():
    vid, wp = synth.make_workload("rgb640x480_k10", width=96, height=72, k=16, n_frames=3)
    out = []
    for form in (pg.PROST_FORM_PASSES, pg.PROST_FORM_PASSES, pg.PROST_FORM_GRID):
        h = pg.prost_init(gpu_params(wp, form=form, seed=3))
        try:
            masks = []
            for t in range(3):
                m = np.empty(vid.P, np.uint8)
                assert pg.prost_step(h, vid.frame(t)[0], m) == pg.PROST_OK
                masks.append(m)
            U = np.empty((vid.m, vid.k), np.float32)
            y = np.empty(vid.k)
            pg.prost_get_subspace(h, U, y)
            out.append((U, y, masks, pg.prost_get_stats(h).form))
        finally:
            pg.prost_destroy(h)
    (Ua, ya, ma, fa), (Ub, yb, mb, fb), (Ug, yg, mg, fg) = out
    assert fa == fb == pg.PROST_FORM_PASSES and fg == pg.PROST_FORM_GRID
    assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
    assert all(np.array_equal(x, z) for x, z in zip(ma, mb))
    # the two forms sum in different orders: the same subspace to FP32 rounding
    assert _angle_max(Ua, Ug) < 1e-5
    assert np.linalg.norm(ya - yg) <= 1e-5 * np.linalg.norm(yg)


def _wide(k=20, **over):
    vid, wp = synth.make_workload("rgb640x480_k10", width=48, height=36, k=k, n_frames=12)
    return vid, dict(wp, **over)


def _sub(h, vid):
    U = np.empty((vid.m, vid.k), np.float32)
    y = np.empty(vid.k)
    pg.prost_get_subspace(h, U, y)
    return U, y


@pytest.mark.parametrize("k", [17, 32])
def test_initial_subspace_roundtrip_and_rank_check(k):
    vid, wp = _wide(k)
    hs = [pg.prost_init(gpu_params(wp, seed=s)) for s in (1, 1, 2)]
    try:
        Us = [_sub(h, vid) for h in hs]
        for U, y in Us:
            np.testing.assert_allclose(U.T.astype(np.float64) @ U, np.eye(k), atol=2e-6)
            assert np.all(y == 0)
        assert np.array_equal(Us[0][0], Us[1][0]) and not np.allclose(Us[0][0], Us[2][0])
        U0 = synth.random_orthonormal(vid.m, k, 5).astype(np.float32)
        y0 = np.arange(1.0, k + 1)
        pg.prost_set_subspace(hs[0], U0, y0)
        U, y = _sub(hs[0], vid)
        np.testing.assert_allclose(U, U0, atol=1e-6)
        np.testing.assert_allclose(U.astype(np.float64) @ y, U0.astype(np.float64) @ y0, atol=1e-5)
        U0[:, 3] = 0.0
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_set_subspace(hs[1], U0)
        assert ei.value.code == pg.PROST_ENOTSPD
    finally:
        for h in hs:
            pg.prost_destroy(h)


def test_host_device_and_pipelined_paths_agree_bit_for_bit():
    vid, wp = _wide(20)
    host = [np.ascontiguousarray(vid.frame(t)[0]) for t in range(8)]
    pinned = [torch.from_numpy(f).pin_memory() for f in host]
    a, b, c = (pg.prost_init(gpu_params(wp, seed=3)) for _ in range(3))
    try:
        ma, mb, mc = [], [], []
        for t in range(8):
            m = np.empty(vid.P, np.uint8)
            assert pg.prost_step(a, host[t], m) == pg.PROST_OK
            ma.append(m)
            fd = torch.from_numpy(host[t]).cuda()
            md = torch.empty(vid.P, dtype=torch.uint8, device="cuda")
            pg.prost_step(b, fd, md)
            mb.append(md)
        assert pg.prost_sync(b) == pg.PROST_OK
        outs = [torch.empty(vid.P, dtype=torch.uint8).pin_memory() for _ in range(8)]
        for t in range(8):
            pg.prost_step_async(c, pinned[t], outs[t])
            if t >= 1:
                assert pg.prost_wait(c) == pg.PROST_OK
        assert pg.prost_wait(c) == pg.PROST_OK
        for t in range(8):
            assert np.array_equal(ma[t], mb[t].cpu().numpy()) and np.array_equal(ma[t], outs[t].numpy())
        (Ua, ya), (Ub, yb), (Uc, yc) = _sub(a, vid), _sub(b, vid), _sub(c, vid)
        assert np.array_equal(Ua, Ub) and np.array_equal(Ua, Uc)
        assert np.array_equal(ya, yb) and np.array_equal(ya, yc)
    finally:
        for h in (a, b, c):
            pg.prost_destroy(h)


def test_checkpoint_and_injection_limits_of_the_passes_form():
    vid, wp = _wide(24)
    a = pg.prost_init(gpu_params(wp, seed=4))
    b = pg.prost_init(gpu_params(wp, seed=9))
    try:
        for t in range(3):
            assert pg.prost_step(a, vid.frame(t)[0], np.empty(vid.P, np.uint8)) == pg.PROST_OK
        state = pg.prost_get_state(a)
        pg.prost_set_state(b, state)
        for t in range(3, 6):
            f = vid.frame(t)[0]
            ma, mb = np.empty(vid.P, np.uint8), np.empty(vid.P, np.uint8)
            assert pg.prost_step(a, f, ma) == pg.PROST_OK and pg.prost_step(b, f, mb) == pg.PROST_OK
            assert np.array_equal(ma, mb)
        (Ua, ya), (Ub, yb) = _sub(a, vid), _sub(b, vid)
        assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
        # the passes form has no grid barrier to skew or stall
        for call in (lambda: pg.prost_inject_barrier_skew(a, -1), lambda: pg.prost_inject_wait_timeout(a, 0, 1000)):
            with pytest.raises(pg.ProstError) as ei:
                call()
            assert ei.value.code == pg.PROST_EINVAL
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)
