"""Property tests of the oracle over random small problems: invariants the
mathematics fixes for every input, beyond the seeded cases of the pins.
Examples are drawn by hypothesis with a fixed derandomised seed; the module is
skipped where hypothesis is not installed."""

import numpy as np
import pytest

import oracle
import synth

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = settings(max_examples=40, deadline=None, derandomize=True)


def _prm(W, H, C, k, **kw):
    base = dict(p=0.25, mu=0.05, delta=0.35, omega=5e-5, t_init=5e-3, t_min=1e-4,
                i_init=100, n_cg=5, in_scale=1.0, in_offset=0.0)
    base.update(kw)
    return oracle.params(W, H, C, k, **base)


def _problem(seed, W, H, C, k, outliers):
    rng = np.random.default_rng(seed)
    m, P = W * H * C, W * H
    U = synth.random_orthonormal(m, k, rng)
    x = U @ (rng.standard_normal(k) * 2.0) + 0.02 * rng.standard_normal(m)
    bad = rng.random(m) < outliers
    x[bad] += rng.uniform(-2, 2, int(bad.sum()))
    labels = (rng.random(P) < 0.2).astype(np.uint8)
    return rng, U, x, labels


shapes = st.tuples(st.integers(2, 9), st.integers(2, 7), st.sampled_from([1, 3]), st.integers(1, 4))


@SETTINGS
@given(seed=st.integers(0, 2 ** 31), shape=shapes, p=st.floats(0.05, 2.0), mu=st.floats(1e-3, 1.0))
def test_cost_is_invariant_under_a_change_of_basis(seed, shape, p, mu):
    # the cost depends on U and y only through U y (Eq. spcacost)
    W, H, C, k = shape
    rng, U, x, labels = _problem(seed, W, H, C, k, 0.1)
    prm = _prm(W, H, C, k, p=p, mu=mu, omega=0.3)
    w = oracle.weights(prm, labels)
    y = rng.standard_normal(k)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    assert oracle.cost(prm, U @ Q, Q.T @ y, x, w) == pytest.approx(oracle.cost(prm, U, y, x, w), rel=1e-12)


@SETTINGS
@given(seed=st.integers(0, 2 ** 31), shape=shapes, p=st.floats(0.05, 2.0), mu=st.floats(1e-3, 1.0),
       n_cg=st.integers(1, 10))
def test_cg_never_increases_the_cost(seed, shape, p, mu, n_cg):
    # the majorise-minimise line step is a descent step for every p <= 2
    W, H, C, k = shape
    rng, U, x, labels = _problem(seed, W, H, C, k, 0.2)
    prm = _prm(W, H, C, k, p=p, mu=mu, n_cg=n_cg, omega=0.3)
    w = oracle.weights(prm, labels)
    y, tr = oracle.cg(prm, U, x, w, rng.standard_normal(k) * 3)
    c = np.array(tr.cost[:n_cg + 1])
    assert np.all(np.diff(c) <= 1e-12 * c[0])
    assert oracle.cost(prm, U, y, x, w) == pytest.approx(c[-1], rel=1e-12)


@SETTINGS
@given(seed=st.integers(0, 2 ** 31), shape=shapes, t=st.floats(0.0, 10.0))
def test_geodesic_step_stays_on_the_stiefel_manifold(seed, shape, t):
    # U(t) has orthonormal columns for every t (Eq. geodesic), and U(0) = U
    W, H, C, k = shape
    rng, U, x, labels = _problem(seed, W, H, C, k, 0.1)
    prm = _prm(W, H, C, k, omega=0.3)
    w = oracle.weights(prm, labels)
    y = rng.standard_normal(k)
    e = oracle.eta(prm, oracle.residual(U, y, x), w)
    Ut, _ = oracle.grassmann_step(prm, U, y, e, t)
    np.testing.assert_allclose(Ut.T @ Ut, np.eye(k), atol=1e-12)
    U0, _ = oracle.grassmann_step(prm, U, y, e, 0.0)
    np.testing.assert_allclose(U0, U, atol=1e-14)


@SETTINGS
@given(seed=st.integers(0, 2 ** 31), shape=shapes, scale=st.floats(0.1, 10.0))
def test_reorthonormalisation_keeps_the_span_and_u_y(seed, shape, scale):
    W, H, C, k = shape
    m = W * H * C
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * scale
    y = rng.standard_normal(k)
    Un, yn = oracle.reorthonormalize(A, y)
    np.testing.assert_allclose(Un.T @ Un, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(Un @ yn, A @ y, rtol=1e-10, atol=1e-12 * np.abs(A @ y).max())
    # same column space: the projector onto it is unchanged
    Qa, _ = np.linalg.qr(A)
    np.testing.assert_allclose(Un @ Un.T, Qa @ Qa.T, atol=1e-12)


@SETTINGS
@given(seed=st.integers(0, 2 ** 31), shape=shapes, d1=st.floats(0.01, 1.0), d2=st.floats(0.01, 1.0))
def test_labels_shrink_as_the_threshold_grows(seed, shape, d1, d2):
    # F_q = [max_c |r_cq| >= delta]: a larger delta labels a subset of the pixels
    W, H, C, k = shape
    rng, U, x, _ = _problem(seed, W, H, C, k, 0.3)
    y = rng.standard_normal(k)
    lo, hi = min(d1, d2), max(d1, d2)
    lab_lo, mx, n_lo = oracle.labels(_prm(W, H, C, k, delta=lo), U, y, x)
    lab_hi, _, n_hi = oracle.labels(_prm(W, H, C, k, delta=hi), U, y, x)
    assert np.all(lab_hi <= lab_lo) and n_hi <= n_lo
    r = np.abs(x - U @ y).reshape(C, W * H).max(axis=0)
    np.testing.assert_allclose(mx, r, rtol=1e-12, atol=1e-15)
    assert np.array_equal(lab_lo, (r >= lo).astype(np.uint8))
