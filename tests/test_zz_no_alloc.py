"""prost_cost_grad_static(): the entry point for callers that cannot
allocate device memory (real-time loops that allow no cudaMalloc after
start-up, because it can synchronise the device and has no latency bound;
plug-ins whose host owns all device memory and passes them only their
buffers).  It keeps its reduction scratch in a static device array inside the
library, so it is checked here against what the allocating path (prost_init /
prost_step) reports for the same frame: the cost and the gradient norm at the
warm-start coefficients.  Two calls run back to back to show that the shared
static scratch is cleared between calls.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""

import numpy as np
import pytest

import oracle
import synth
import paper_1302_2073_gb300 as pg
from parity import COST_RTOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _allocating_path(wp, U0, y, labels, frame):
    """Cost and |gradient| at y from the handle-based path (first CG pass)."""
    h = pg.prost_init(pg.make_params(**wp))
    try:
        pg.prost_set_subspace(h, U0, y)
        pg.prost_set_labels(h, labels)
        mask = np.empty(labels.size if labels is not None else U0.shape[0] // wp["channels"],
                        dtype=np.uint8)
        assert pg.prost_step(h, frame, mask) == pg.PROST_OK
        st = pg.prost_get_stats(h)
        return st.cost[0], st.gnorm[0], mask
    finally:
        pg.prost_destroy(h)


def test_static_scratch_entry_matches_allocating_path_twice():
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA GPU")
    vid, wp = synth.make_workload("rgb640x480_k10", width=320, height=240, n_frames=3)
    rng = np.random.default_rng(21)
    U0 = synth.random_orthonormal(vid.m, vid.k, rng).astype(np.float32)
    y = rng.standard_normal(vid.k) * 20.0
    prm = pg.make_params(**wp)
    prm_o = oracle.params(**wp)

    U_dev = torch.from_numpy(U0).cuda()
    out = torch.empty(vid.k + 1, dtype=torch.float64, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")

    labels = None
    for t in range(2):  # two calls in a row, different frames and weights
        frame, _ = vid.frame(t)
        cost_ref, gnorm_ref, mask = _allocating_path(wp, U0, y, labels, frame)
        out.fill_(float("nan"))
        status.fill_(-99)
        lab_dev = None if labels is None else torch.from_numpy(labels).cuda()
        pg.prost_cost_grad_static(prm, U_dev, y, torch.from_numpy(frame).cuda(), lab_dev,
                                  out, status)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        assert int(status.item()) == pg.PROST_OK
        assert abs(res[0] - cost_ref) <= COST_RTOL * abs(cost_ref)
        assert abs(np.linalg.norm(res[1:]) - gnorm_ref) <= COST_RTOL * gnorm_ref
        # the gradient vector itself against the FP64 oracle: U^T eta at (U0, y)
        x = oracle.preprocess(prm_o, frame)
        w = oracle.weights(prm_o, labels)
        g_o = oracle.ut(U0.astype(np.float64),
                        oracle.eta(prm_o, oracle.residual(U0.astype(np.float64), y, x), w))
        assert np.linalg.norm(res[1:] - g_o) <= COST_RTOL * np.linalg.norm(g_o)
        labels = mask  # the second call weights the first frame's foreground by omega
    assert labels.any()


def test_static_scratch_entry_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA GPU")
    vid, wp = synth.make_workload("gray160x120_k5", width=32, height=24, n_frames=1)
    bad = pg.make_params(**dict(wp, k=pg.PROST_STATIC_MAX_K + 1))
    U = torch.zeros((vid.m, pg.PROST_STATIC_MAX_K + 1), dtype=torch.float32, device="cuda")
    out = torch.empty(pg.PROST_STATIC_MAX_K + 2, dtype=torch.float64, device="cuda")
    f = torch.zeros(vid.m, dtype=torch.float32, device="cuda")
    with pytest.raises(pg.ProstError) as ei:
        pg.prost_cost_grad_static(bad, U, [0.0] * (pg.PROST_STATIC_MAX_K + 1), f, None, out)
    assert ei.value.code == pg.PROST_EINVAL
