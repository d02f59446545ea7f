"""The bfloat16 subspace storage (PROST_BF16) against the FP64 oracle.

Storage in bfloat16 is not in the paper.  Its results differ from the FP32
storage by the rounding of the stored rows (about 2^-9 of each entry, renewed
unbiasedly at every update), so these tests bound the error rather than
demand parity: a single teacher-forced step (relative error of the residual and
the cost, mask disagreement), a free-running trajectory (principal angle to the
oracle's subspace, mask disagreement over the frames), orthonormality of the
exported subspace, and bit-identical resumption (the stochastic rounding is a
counter-based function of the seed, the frame and the entry)."""

import numpy as np
import pytest

import oracle
import synth
import paper_1302_2073_gb300 as pg
from parity import gpu_params, matched_start, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# bounds on the measured error of the bfloat16 storage (see the module
# docstring; the FP32 storage meets the parity tolerances of tests/parity.py)
STEP_RES_RTOL = 1e-3   # measured 2.9e-5 (160x120 RGB, k = 10)
STEP_COST_RTOL = 1e-4  # measured 5.1e-8
STEP_MASK_FRAC = 2e-3  # measured 0
# over 200 free-running frames the rounding noise of the stored rows adds up as
# a random walk (about half an ulp times the square root of the frame count)
# in the directions the data does not currently excite: measured 3.0e-2 rad,
# against 3.7e-7 rad for the FP32 storage; the masks barely notice (4.7e-5)
RUN_ANGLE = 1e-1
RUN_MASK_FRAC = 2e-3


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _angle(A, B):
    qa, _ = np.linalg.qr(np.asarray(A, np.float64))
    qb, _ = np.linalg.qr(np.asarray(B, np.float64))
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


@pytest.mark.parametrize("k", [1, 5, 10, 15, 16])
def test_bf16_initial_subspace_is_orthonormal(k):
    vid = synth.SyntheticVideo(40, 30, 3, k, n_frames=1, seed=3, dtype="u8")
    wp = synth.video._params(vid.m, k, "u8")
    wp.update(width=40, height=30, channels=3, frame_dtype="u8")
    h = pg.prost_init(gpu_params(wp, u_dtype="bf16"))
    try:
        U = np.empty((vid.m, k), np.float32)
        pg.prost_get_subspace(h, U, np.empty(k))
    finally:
        pg.prost_destroy(h)
    np.testing.assert_allclose(U.T.astype(np.float64) @ U, np.eye(k), atol=5e-6)


@pytest.mark.parametrize("k,w,h,form", [
    (10, 160, 120, pg.PROST_FORM_AUTO),       # the resident form, every row in shared memory
    (15, 160, 120, pg.PROST_FORM_AUTO),       # the streaming form
    (10, 1280, 720, pg.PROST_FORM_RESIDENT),  # the resident form with rows streaming from L2
])
def test_bf16_teacher_forced_step(k, w, h, form):
    vid, wp = synth.make_workload("rgb640x480_k10", width=w, height=h, n_frames=4, k=k)
    prm_o = oracle_params(wp)
    st = oracle.initial_state(synth.random_orthonormal(vid.m, vid.k, 21), vid.P)
    for t in range(3):
        oracle.frame_step(prm_o, st, vid.frame(t)[0])
    f, _ = vid.frame(3)
    U32, U64, y64 = matched_start(st.U, st.y)
    h = pg.prost_init(gpu_params(wp, u_dtype="bf16", form=form))
    try:
        pg.prost_set_subspace(h, U32, y64)
        pg.prost_set_labels(h, st.labels)
        pg.prost_set_frame_index(h, st.i)
        mask = np.empty(vid.P, np.uint8)
        bg = np.empty(vid.m, np.float32)
        assert pg.prost_step(h, f, mask, bg) == pg.PROST_OK
        stats = pg.prost_get_stats(h)
    finally:
        pg.prost_destroy(h)
    ref = oracle.OracleState(U64.copy(), y64.copy(), st.labels.copy(), st.i)
    res = oracle.frame_step(prm_o, ref, f)
    x = f.reshape(-1).astype(np.float64) * wp["in_scale"] - wp["in_offset"]
    r_gpu = x - (bg.astype(np.float64) - wp["in_offset"])
    res_rel = np.linalg.norm(r_gpu - res.residual) / np.linalg.norm(res.residual)
    cost_rel = abs(stats.cost[0] - res.trace.cost[0]) / res.trace.cost[0]
    mask_frac = float((mask != res.labels).mean())
    print(f"bf16 step k={k}: residual rel {res_rel:.2e}, cost rel {cost_rel:.2e}, mask disagreement {mask_frac:.2e}")
    assert res_rel < STEP_RES_RTOL and cost_rel < STEP_COST_RTOL and mask_frac < STEP_MASK_FRAC


def _free_run(wp, vid, n, u_dtype, seed=5):
    prm_o = oracle_params(wp)
    U32, U64, y64 = matched_start(synth.random_orthonormal(vid.m, vid.k, seed), np.zeros(vid.k))
    st = oracle.OracleState(U64.copy(), y64.copy(), np.zeros(vid.P, np.uint8), 0)
    h = pg.prost_init(gpu_params(wp, u_dtype=u_dtype))
    dis = []
    try:
        pg.prost_set_subspace(h, U32)
        m = np.empty(vid.P, np.uint8)
        for t in range(n):
            f, _ = vid.frame(t)
            assert pg.prost_step(h, f, m) == pg.PROST_OK
            res = oracle.frame_step(prm_o, st, f, want_residual=False)
            dis.append(float((m != res.labels).mean()))
        Ug = np.empty((vid.m, vid.k), np.float32)
        pg.prost_get_subspace(h, Ug, np.empty(vid.k))
    finally:
        pg.prost_destroy(h)
    return _angle(Ug, st.U), float(np.mean(dis)), float(np.max(dis))


def test_bf16_free_running_trajectory_tracks_the_oracle():
    vid, wp = synth.make_workload("gray160x120_k5", n_frames=200)
    a16, m16, x16 = _free_run(wp, vid, 200, "bf16")
    a32, m32, x32 = _free_run(wp, vid, 200, "f32")
    print(f"200 frames: bf16 angle {a16:.2e} rad, mask {m16:.2e} (max {x16:.2e}); "
          f"fp32 angle {a32:.2e} rad, mask {m32:.2e}")
    assert a16 < RUN_ANGLE and m16 < RUN_MASK_FRAC
    assert a32 < 1e-4


def test_bf16_checkpoint_resumes_bit_identically():
    vid = synth.SyntheticVideo(48, 36, 3, 6, n_frames=12, fg_fraction=0.05, seed=8, dtype="u8")
    wp = synth.video._params(vid.m, vid.k, "u8")
    wp.update(width=48, height=36, channels=3, frame_dtype="u8")
    frames = vid.frames(0, 12)
    a = pg.prost_init(gpu_params(wp, u_dtype="bf16"))
    b = pg.prost_init(gpu_params(wp, u_dtype="bf16"))
    try:
        m = np.empty(vid.P, np.uint8)
        for t in range(6):
            pg.prost_step(a, frames[t], m)
        ck = pg.prost_get_state(a)
        for t in range(6, 12):
            pg.prost_step(a, frames[t], m)
        pg.prost_set_state(b, ck)
        for t in range(6, 12):
            pg.prost_step(b, frames[t], m)
        Ua, Ub = np.empty((vid.m, 6), np.float32), np.empty((vid.m, 6), np.float32)
        ya, yb = np.empty(6), np.empty(6)
        pg.prost_get_subspace(a, Ua, ya)
        pg.prost_get_subspace(b, Ub, yb)
    finally:
        pg.prost_destroy(a)
        pg.prost_destroy(b)
    assert np.array_equal(Ua, Ub) and np.array_equal(ya, yb)
