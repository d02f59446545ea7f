"""GPU pre- and post-processing (Section 3.4) against the FP64 oracle, through
the C ABI: area resampling with the running mean/deviation normalisation
(through and after the initialisation phase), the 3 x 3 mask median
(bit-exact), and the paper's whole per-frame pipeline (pre-processing,
tracker, median)."""

import numpy as np
import pytest

import oracle
import synth
import paper_1302_2073_gb300 as pg
from oracle import prepost as pp
from parity import MASK_BAND, gpu_params, matched_start, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 resampling (footprint weights, sums of at most a few hundred terms) and
# FP32 running mean: relative to the deviation, well inside 1e-5
PRE_ATOL = 1e-5


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


@pytest.mark.parametrize("w_in,h_in,C,w_out,h_out,dtype", [
    (640, 480, 3, 160, 120, "u8"),   # the paper's resampling of a 640x480 stream
    (100, 75, 3, 37, 29, "u8"),      # non-integer ratios, ragged footprints
    (1366, 768, 3, 160, 120, "u8"),  # large non-integer ratios: exact integer footprints
    (33, 21, 1, 40, 30, "f32"),      # upsampling, float frames
])
def test_pre_processing_through_and_after_the_phase(w_in, h_in, C, w_out, h_out, dtype):
    rng = np.random.default_rng(w_in + h_in)
    n, i_init = 7, 4
    if dtype == "u8":
        frames = rng.integers(0, 256, size=(n, C, h_in, w_in)).astype(np.uint8)
    else:
        frames = rng.random((n, C, h_in, w_in)).astype(np.float32)
    ref = pp.RunningNorm((C, h_out, w_out), i_init)
    p = pg.prost_pre_init(w_in, h_in, C, w_out, h_out, dtype, i_init)
    try:
        out = torch.empty((C, h_out, w_out), dtype=torch.float32, device="cuda")
        for t in range(n):
            pg.prost_pre_apply(p, torch.from_numpy(frames[t]).cuda(), out)
            want = ref.apply(pp.resample_area(frames[t], w_out, h_out))
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=1e-5, atol=PRE_ATOL)
        mean = np.empty((C, h_out, w_out), np.float32)
        sd, cnt = pg.prost_pre_get_stats(p, mean)
    finally:
        pg.prost_pre_destroy(p)
    assert cnt == i_init
    assert sd == pytest.approx(ref.std(), rel=1e-6)
    np.testing.assert_allclose(mean, ref.mean, rtol=1e-5, atol=1e-4)


def test_pre_processing_host_buffers():
    rng = np.random.default_rng(9)
    f = rng.integers(0, 256, size=(3, 48, 64)).astype(np.uint8)
    p = pg.prost_pre_init(64, 48, 3, 16, 12, "u8", 10)
    try:
        out = np.empty((3, 12, 16), np.float32)
        pg.prost_pre_apply(p, f, out)
    finally:
        pg.prost_pre_destroy(p)
    want = pp.RunningNorm((3, 12, 16), 10).apply(pp.resample_area(f, 16, 12))
    np.testing.assert_allclose(out, want, rtol=1e-5, atol=PRE_ATOL)


@pytest.mark.parametrize("w,h,p1", [(160, 120, 0.1), (37, 29, 0.5), (1, 1, 1.0), (1, 17, 0.5), (64, 1, 0.5),
                                    (640, 480, 0.08)])
def test_median_is_bit_exact(w, h, p1):
    rng = np.random.default_rng(w * 1000 + h)
    m = (rng.random((h, w)) < p1).astype(np.uint8) * rng.integers(1, 256, size=(h, w)).astype(np.uint8)
    want = pp.median3x3_mask(m)
    d_in = torch.from_numpy(m).cuda()
    d_out = torch.empty_like(d_in)
    pg.prost_median3x3(d_in, d_out, w, h)
    np.testing.assert_array_equal(d_out.cpu().numpy(), want)
    h_out = np.empty_like(m)
    pg.prost_median3x3(m, h_out, w, h)
    np.testing.assert_array_equal(h_out, want)


def test_median_rejects_in_place_and_bad_sizes():
    d = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(pg.ProstError):
        pg.prost_median3x3(d, d, 4, 4)
    with pytest.raises(pg.ProstError):
        pg.prost_median3x3(d, torch.empty_like(d), 0, 4)


def test_pipeline_pre_tracker_median_against_the_oracle():
    """640x480 RGB frames -> 160x120 normalised -> one tracker step from a
    common state -> 3 x 3 median, both sides; masks equal except within one
    pixel of a pixel whose oracle residual lies within the band of the
    threshold."""
    vid, _ = synth.make_workload("rgb640x480_k10", n_frames=3)
    w, h = 160, 120
    wp = synth.video._params(3 * w * h, 10, "f32")
    wp.update(width=w, height=h, channels=3, frame_dtype="f32", in_scale=1.0, in_offset=0.0)
    prm_o = oracle_params(wp)
    ref_pre = pp.RunningNorm((3, h, w), i_init=100)
    p = pg.prost_pre_init(640, 480, 3, w, h, "u8", 100)
    hdl = pg.prost_init(gpu_params(wp))
    try:
        U32, U64, y64 = matched_start(synth.random_orthonormal(3 * w * h, 10, 4), np.zeros(10))
        st = oracle.OracleState(U64.copy(), y64.copy(), np.zeros(w * h, np.uint8), 0)
        pg.prost_set_subspace(hdl, U32)
        x = torch.empty((3, h, w), dtype=torch.float32, device="cuda")
        mask = torch.empty(w * h, dtype=torch.uint8, device="cuda")
        med = torch.empty_like(mask)
        for t in range(3):
            f, _ = vid.frame(t)
            pg.prost_pre_apply(p, torch.from_numpy(f).cuda(), x)
            xo = ref_pre.apply(pp.resample_area(f, w, h))
            np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=1e-5, atol=PRE_ATOL)
            # both trackers from the same state and the same (oracle) input
            Ug = np.empty((3 * w * h, 10), np.float32)
            yg = np.empty(10)
            pg.prost_get_subspace(hdl, Ug, yg)
            U32, U64, y64 = matched_start(st.U, st.y)
            pg.prost_set_subspace(hdl, U32, y64)
            pg.prost_set_labels(hdl, st.labels)
            pg.prost_set_frame_index(hdl, st.i)
            st = oracle.OracleState(U64.copy(), y64.copy(), st.labels.copy(), st.i)
            xin = torch.from_numpy(xo.astype(np.float32)).cuda()
            pg.prost_step(hdl, xin, mask)
            pg.prost_sync(hdl)
            res = oracle.frame_step(prm_o, st, xo.astype(np.float32))
            pg.prost_median3x3(mask, med, w, h)
            want = pp.median3x3_mask(res.labels.reshape(h, w))
            got = med.cpu().numpy().reshape(h, w)
            # excused: pixels within one pixel of a near-threshold residual
            r = np.abs(res.residual.reshape(3, h * w)).max(axis=0).reshape(h, w)
            near = np.abs(r - wp["delta"]) <= MASK_BAND
            near = np.pad(near, 1, mode="edge")
            band = np.zeros((h, w), bool)
            for dy in range(3):
                for dx in range(3):
                    band |= near[dy:dy + h, dx:dx + w]
            assert ((got != want) & ~band).sum() == 0
    finally:
        pg.prost_destroy(hdl)
        pg.prost_pre_destroy(p)


@pytest.mark.parametrize("cut", [0, 3, 6, 9])
def test_pre_processing_resumes_bit_identically_from_a_checkpoint(cut):
    """A pre-processor restored from a checkpoint taken after `cut` frames
    (before, inside and after its 6-frame initialisation phase) gives the same
    output bits as the one that never stopped."""
    rng = np.random.default_rng(17)
    frames = [rng.integers(0, 256, size=(3, 96, 128)).astype(np.uint8) for _ in range(11)]
    a = pg.prost_pre_init(128, 96, 3, 40, 30, "u8", 6)
    b = pg.prost_pre_init(128, 96, 3, 40, 30, "u8", 6)
    try:
        out_a = []
        ck = None
        for t, f in enumerate(frames):
            if t == cut:
                ck = pg.prost_pre_get_state(a)
            o = np.empty(3 * 30 * 40, np.float32)
            pg.prost_pre_apply(a, f, o)
            out_a.append(o)
        if ck is None:
            ck = pg.prost_pre_get_state(a)
        pg.prost_pre_set_state(b, ck)
        for t in range(cut, len(frames)):
            o = np.empty(3 * 30 * 40, np.float32)
            pg.prost_pre_apply(b, frames[t], o)
            assert np.array_equal(o, out_a[t]), t
        ma, mb = np.empty(3 * 30 * 40, np.float32), np.empty(3 * 30 * 40, np.float32)
        sa, sb = pg.prost_pre_get_stats(a, ma), pg.prost_pre_get_stats(b, mb)
        assert np.array_equal(ma, mb) and sa == sb
    finally:
        pg.prost_pre_destroy(a)
        pg.prost_pre_destroy(b)


def test_pre_processing_checkpoint_refuses_other_parameters():
    a = pg.prost_pre_init(128, 96, 3, 40, 30, "u8", 6)
    b = pg.prost_pre_init(128, 96, 3, 40, 30, "u8", 5)
    try:
        ck = pg.prost_pre_get_state(a)
        with pytest.raises(pg.ProstError) as ei:
            pg.prost_pre_set_state(b, ck)
        assert ei.value.code == pg.PROST_EINVAL
        with pytest.raises(pg.ProstError):
            pg.prost_pre_set_state(a, ck[:-4])
    finally:
        pg.prost_pre_destroy(a)
        pg.prost_pre_destroy(b)
