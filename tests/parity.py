"""Helpers of the GPU-vs-oracle parity tests (teacher forcing: both sides
start a frame from the same state and advance it once)."""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle
import paper_1302_2073_gb300 as pg

# Tolerances (FP32 GPU vs FP64 oracle).  The residual and cost bound is the
# stated acceptance bound; masks may differ only at pixels whose FP64 maximum
# residual lies within MASK_BAND of delta.
RES_RTOL = 1e-4
COST_RTOL = 1e-4
MASK_BAND = 1e-6
# FP32 storage of U (relative rounding 6e-8 per entry) and FP32 per-row
# arithmetic bound the coefficient and subspace differences well below these.
Y_RTOL = 1e-5
U_RTOL = 1e-5
THETA_RTOL = 1e-4
# The step size t = max(exp(-tau i) t_init, t_min) of Section 3.3 enters only
# through theta = sigma t, an FP32 product, so the kernel forms t to FP32
# accuracy: the FP32 exponential (2 ulp) of the reduced argument (rounded to
# FP32) scaled by t_init (rounded to FP32), about 4e-7 relative at most.
T_RTOL = 1e-6
# Step 2 normalises pi(eta) (Eq. svd).  The FP32 pass resolves pi(eta) only to
# about 1e-7 |eta| (the rounding of the residual and of u^T g per entry), so
# where the oracle's |pi(eta)| lies below PI_BAND |eta| rounding decides the
# step on both sides: either skip decision is accepted there, and theta is
# compared absolutely, |theta_gpu - theta_oracle| <= 2 PI_BAND |eta| |y| t.
PI_BAND = 1e-5


def _rel(a, b):
    """|a - b| / |b|, 0 when both are zero (a degenerate reference)."""
    nb = float(np.linalg.norm(b))
    d = float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)))
    if nb > 0.0:
        return d / nb
    return 0.0 if d == 0.0 else float("inf")


def oracle_eta_norm(prm_o, U64, y64, labels, frame):
    """|eta| at the oracle's final y of the frame (Section 3.3)."""
    x = oracle.preprocess(prm_o, frame)
    w = oracle.weights(prm_o, labels)
    y, _ = oracle.cg(prm_o, U64, x, w, y64)
    return float(np.linalg.norm(oracle.eta(prm_o, oracle.residual(U64, y, x), w)))


def oracle_params(wp: dict):
    return oracle.params(**wp)


def gpu_params(wp: dict, **over):
    d = dict(wp)
    d.update(over)
    return pg.make_params(**d)


@dataclass
class GpuStep:
    mask: np.ndarray
    background: np.ndarray
    U: np.ndarray
    y: np.ndarray
    stats: object
    status: int


def matched_start(U, y):
    """The state both sides start from: FP32 rounding of U, re-orthonormalised
    (what the GPU stores), and y transformed so that U y is kept."""
    U32 = np.ascontiguousarray(U, dtype=np.float32)
    U64, y64 = oracle.reorthonormalize(U32.astype(np.float64), np.asarray(y, dtype=np.float64))
    return U32, U64, y64


def gpu_step_from(h, U32, y, labels, i, frame, device=True, torch=None):
    """Hand the GPU tracker a state, run one frame, read everything back."""
    m, k = U32.shape
    P = labels.size
    pg.prost_set_subspace(h, U32, np.ascontiguousarray(y, dtype=np.float64))
    pg.prost_set_labels(h, np.ascontiguousarray(labels, dtype=np.uint8))
    pg.prost_set_frame_index(h, i)
    if device:
        f = torch.from_numpy(np.ascontiguousarray(frame)).cuda()
        mask = torch.empty(P, dtype=torch.uint8, device="cuda")
        bg = torch.empty(m, dtype=torch.float32, device="cuda")
        pg.prost_step(h, f, mask, bg)
        status = pg.prost_sync(h)
        mask, bg = mask.cpu().numpy(), bg.cpu().numpy()
    else:
        mask = np.empty(P, dtype=np.uint8)
        bg = np.empty(m, dtype=np.float32)
        status = pg.prost_step(h, np.ascontiguousarray(frame), mask, bg)
    stats = pg.prost_get_stats(h)
    Ug = np.empty((m, k), dtype=np.float32)
    yg = np.empty(k)
    pg.prost_get_subspace(h, Ug, yg)
    return GpuStep(mask, bg, Ug, yg, stats, status)


def compare_step(prm_o, wp, U64, y64, labels, i, frame, g: GpuStep, n_cg=None, pi_band=False):
    """Run the oracle from the same state and assert parity; returns a dict of
    the measured errors.  pi_band: apply the PI_BAND rule to Step 2 (needs one
    more oracle CG run for |eta|)."""
    eta_n = oracle_eta_norm(prm_o, U64, y64, labels, frame) if pi_band else None
    st = oracle.OracleState(U64.copy(), y64.copy(), labels.copy(), i)
    res = oracle.frame_step(prm_o, st, frame)
    tr = res.trace
    n = prm_o.n_cg if n_cg is None else n_cg
    x = oracle.preprocess(prm_o, frame)
    P = labels.size
    C = x.size // P
    err = {}
    cg = np.array([g.stats.cost[j] for j in range(n + 1)])
    co = np.array([tr.cost[j] for j in range(n + 1)])
    err["cost"] = float(np.max(np.abs(cg - co) / np.abs(co)))
    assert err["cost"] <= COST_RTOL, (cg, co)
    err["y"] = _rel(g.y, st.y)
    assert err["y"] <= Y_RTOL, (g.y, st.y)
    r_gpu = x - (g.background.astype(np.float64) - prm_o.in_offset)
    err["res"] = _rel(r_gpu, res.residual)
    assert err["res"] <= RES_RTOL
    if pi_band and tr.pi_norm < PI_BAND * eta_n:
        # rounding decides the step on both sides
        err["theta_abs"] = abs(g.stats.theta - tr.theta)
        assert err["theta_abs"] <= 2.0 * PI_BAND * eta_n * tr.y_norm * tr.t, (g.stats.theta, tr.theta)
    else:
        if tr.updated:
            err["theta"] = abs(g.stats.theta - tr.theta) / tr.theta
            assert err["theta"] <= THETA_RTOL, (g.stats.theta, tr.theta)
        assert g.stats.updated == tr.updated
    err["U"] = _rel(g.U, st.U)
    assert err["U"] <= U_RTOL
    maxres = np.abs(res.residual.reshape(C, P)).max(0)
    diff = g.mask != res.labels
    excused = np.abs(maxres - prm_o.delta) <= MASK_BAND
    err["mask_diff"] = int(diff.sum())
    err["mask_unexcused"] = int((diff & ~excused).sum())
    assert err["mask_unexcused"] == 0, np.nonzero(diff & ~excused)[0][:10]
    assert abs(int(g.stats.n_foreground) - int(tr.n_foreground)) <= int(diff.sum())
    assert g.stats.frames == i + 1
    assert abs(g.stats.t - tr.t) <= T_RTOL * tr.t
    return err, st, res
