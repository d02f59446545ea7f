"""Step 2 at its degenerate and ill-conditioned points: GPU against the FP64
oracle, teacher-forced, through the C ABI.

Step 2 normalises the projected gradient pi(eta) (Eqs. gproject, svd).  The
rank-one step is undefined when |y| = 0 or pi(eta) = 0, and both sides then
skip it (the reading of the degenerate step).  It is ill-conditioned when eta
lies almost wholly in span(U): the identity |pi(eta)|^2 = |eta|^2 - |U^T eta|^2
then cancels, so the kernel forms |pi(eta)| by an explicit pass over U
(stats.pi_explicit).  The cases:

* a zero frame at y = 0: nothing to fit, |y| = 0, Step 2 is skipped;
* a zero frame at y != 0, p = 2, no CG step: r = -U y lies in span(U), so does
  eta = -2 r, and pi(eta) is rounding noise on both sides;
* x = U a rounded to float32, p = 2, no CG step: pi(eta) is the rounding of
  the frame (about 1e-7 |eta|);
* x = U a + noise with |pi(eta)| / |eta| about 1e-3 and 1e-2, in the register
  form (k = 10) and the streaming form (k = 15), float and uint8 frames.

Above PI_BAND |eta| (tests/parity.py) the skip decision must match and theta
agree to 1e-4; below it rounding decides on both sides and theta is compared
absolutely.
"""

import numpy as np
import pytest

import oracle
import synth
import paper_1302_2073_gb300 as pg
from parity import (PI_BAND, compare_step, gpu_params, gpu_step_from, matched_start, oracle_eta_norm,
                    oracle_params)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _wp(width, height, channels, k, frame_dtype="f32", **over):
    """Least-squares setting (p = 2, unit weights) unless overridden; mu is
    explicit because the heuristic delta^2 (1 - p) vanishes at p = 2."""
    wp = dict(width=width, height=height, channels=channels, k=k, p=2.0, mu=0.01, delta=0.35,
              omega=1.0, t_init=0.5, t_min=1e-4, i_init=100, n_cg=0, in_scale=1.0, in_offset=0.5,
              frame_dtype=frame_dtype)
    wp.update(over)
    return wp


def _start(m, k, seed):
    """A seeded float32 subspace and its orthonormal representative U64, the
    basis in which the frames below are built and y is given."""
    rng = np.random.default_rng(seed)
    U32, U64, _ = matched_start(synth.random_orthonormal(m, k, rng), np.zeros(k))
    return rng, U32, U64


FORMS = [pg.PROST_FORM_GRID, pg.PROST_FORM_CLUSTER, pg.PROST_FORM_PASSES, pg.PROST_FORM_RESIDENT]


def _run(wp, U32, U64, y, frame, labels=None, form=pg.PROST_FORM_AUTO):
    """One frame from (U64, y) on both sides: the GPU is handed the float32
    rows with the coefficients that give the same U y, and re-orthonormalises
    them onto U64 itself."""
    P = wp["width"] * wp["height"]
    labels = np.zeros(P, np.uint8) if labels is None else labels
    y_raw = np.linalg.lstsq(U32.astype(np.float64), U64 @ y, rcond=None)[0]
    _, U64, y64 = matched_start(U32, y_raw)
    prm_o = oracle_params(wp)
    h = pg.prost_init(gpu_params(wp, form=form))
    try:
        g = gpu_step_from(h, U32, y_raw, labels, 0, frame, device=True, torch=torch)
        assert g.status == pg.PROST_OK
    finally:
        pg.prost_destroy(h)
    err, st, res = compare_step(prm_o, wp, U64, y64, labels, 0, frame, g, pi_band=True)
    return g, err, res.trace, oracle_eta_norm(prm_o, U64, y64, labels, frame)


def _float_frame(x, wp):
    return (np.asarray(x, np.float64) + wp["in_offset"]).astype(np.float32)


def test_zero_frame_at_zero_coefficients_skips_the_step():
    wp = _wp(64, 48, 3, 10, n_cg=5, p=0.25, mu=0.35 ** 2 * 0.75, omega=5e-5)
    m = 64 * 48 * 3
    _, U32, U64 = _start(m, 10, 1)
    frame = _float_frame(np.zeros(m), wp)  # x = in_scale frame - in_offset = 0 exactly
    g, err, tr, eta_n = _run(wp, U32, U64, np.zeros(10), frame)
    assert tr.updated == 0 and g.stats.updated == 0
    assert g.stats.theta == 0.0 and g.stats.y_norm == 0.0
    assert np.all(g.y == 0.0)
    assert not g.mask.any()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("k", [10, 15])
def test_zero_frame_keeps_eta_in_span(k, form):
    if form == pg.PROST_FORM_RESIDENT and k > 10:
        pytest.skip("the resident form serves k <= 10")
    # r = -U y lies in span(U), so eta = -2 r does, and |U^T eta| = |eta|: the
    # norm identity would leave only rounding, which could take a step along noise
    wp = _wp(64, 48, 3, k)
    m = 64 * 48 * 3
    rng, U32, U64 = _start(m, k, 2 + k)
    y = rng.standard_normal(k) * 3.0
    frame = _float_frame(np.zeros(m), wp)
    g, err, tr, eta_n = _run(wp, U32, U64, y, frame, form=form)
    assert g.stats.pi_explicit == 1
    assert tr.pi_norm < 1e-12 * eta_n
    assert g.stats.pi_norm < 1e-5 * eta_n


@pytest.mark.parametrize("k", [10, 15])
def test_frame_in_span_up_to_its_float32_rounding(k):
    wp = _wp(64, 48, 3, k)
    m = 64 * 48 * 3
    rng, U32, U64 = _start(m, k, 20 + k)
    y0 = rng.standard_normal(k)
    a = y0 + rng.standard_normal(k) * 2.0
    frame = _float_frame(U64 @ a * 0.2, wp)
    g, err, tr, eta_n = _run(wp, U32, U64, y0, frame)
    assert g.stats.pi_explicit == 1
    assert tr.pi_norm < PI_BAND * eta_n  # the band: rounding decides


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("k,ratio", [(10, 1e-3), (10, 1e-2), (15, 1e-3), (15, 1e-2), (7, 3e-2)])
def test_eta_almost_in_span(k, ratio, form):
    if form == pg.PROST_FORM_RESIDENT and k > 10:
        pytest.skip("the resident form serves k <= 10")
    # x = U a + noise: eta = -2 (U (a - y) + noise), pi(eta) = -2 pi(noise)
    wp = _wp(96, 72, 3, k)
    m = 96 * 72 * 3
    rng, U32, U64 = _start(m, k, 40 + k)
    y0 = rng.standard_normal(k) * 2.0
    d = rng.standard_normal(k)
    d *= 4.0 / np.linalg.norm(d)
    noise = rng.standard_normal(m) * (4.0 * ratio / np.sqrt(m))
    frame = _float_frame(U64 @ (y0 + d) + noise, wp)
    g, err, tr, eta_n = _run(wp, U32, U64, y0, frame, form=form)
    got = tr.pi_norm / eta_n
    assert 0.3 * ratio < got < 3.0 * ratio, got
    assert g.stats.pi_explicit == 1
    assert tr.updated == 1 and g.stats.updated == 1
    assert "theta" in err and err["theta"] <= 1e-4
    assert tr.theta > 1e-3  # a step that moves U measurably
    print(k, ratio, err)


@pytest.mark.parametrize("k", [10, 15])
def test_eta_almost_in_span_uint8_frames(k):
    # the off-span part is the uint8 quantisation of the frame itself
    wp = _wp(96, 72, 3, k, frame_dtype="u8", in_scale=1.0 / 255.0, t_init=0.1)
    m = 96 * 72 * 3
    rng, U32, U64 = _start(m, k, 60 + k)
    y0 = rng.standard_normal(k) * 2.0
    d = rng.standard_normal(k)
    d *= 8.0 / np.linalg.norm(d)
    v = U64 @ (y0 + d) + 0.5
    assert 0.0 < v.min() and v.max() < 1.0
    frame = np.round(255.0 * v).astype(np.uint8)
    g, err, tr, eta_n = _run(wp, U32, U64, y0, frame)
    assert tr.pi_norm < 0.1 * eta_n
    assert g.stats.pi_explicit == 1
    assert tr.updated == 1 and g.stats.updated == 1
    assert err["theta"] <= 1e-4


def test_ordinary_frames_take_no_extra_pass():
    # after the CG steps of the benchmark setting the gradient U^T eta is small
    # and eta lies mostly outside span(U): the norm identity serves
    vid, wp = synth.make_workload("rgb640x480_k10", width=96, height=72, n_frames=3)
    prm_o = oracle_params(wp)
    st = oracle.initial_state(synth.random_orthonormal(vid.m, vid.k, 3), vid.P)
    f0, _ = vid.frame(0)
    oracle.frame_step(prm_o, st, f0)
    U32, U64, y64 = matched_start(st.U, st.y)
    f1, _ = vid.frame(1)
    h = pg.prost_init(gpu_params(wp))
    try:
        g = gpu_step_from(h, U32, st.y, st.labels, st.i, f1, device=True, torch=torch)
    finally:
        pg.prost_destroy(h)
    err, _, _ = compare_step(prm_o, wp, U64, y64, st.labels, st.i, f1, g, pi_band=True)
    assert g.stats.pi_explicit == 0
    assert g.stats.pi_norm ** 2 > 0.25 * g.stats.eta_norm ** 2
