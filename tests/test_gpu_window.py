"""The windowed cost and its hand-written adjoint on the GPU, through the C ABI
and torch.autograd: against the FP64 oracle at the measured size (320x240,
n = 64, k = 10, 5 % outliers) and on ragged small cases, against central
differences of the GPU's own cost, and the U-step that consumes the gradient."""

import numpy as np
import pytest

import synth
import paper_1302_2073_gb300 as pg
from oracle import window as wo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 sums of at most a tile's rows or a window's frames per term, then FP64:
# norm-relative errors stay near 1e-6
COST_RTOL = 1e-5
GRAD_RTOL = 1e-5
# per entry: an FP32 sum of n frame terms (dU) or of a tile's rows then FP64
# across tiles (dY), against the largest entry of the gradient
ELEM_RTOL = 1e-5


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")


def _case(m, C, k, n, seed, outliers=0.05, label_frac=0.05):
    rng = np.random.default_rng(seed)
    U0 = synth.random_orthonormal(m, k, rng)
    Y0 = rng.standard_normal((k, n)) * 0.1 * np.sqrt(m / k)
    X = (U0 @ Y0).T
    out = rng.random((n, m)) < outliers
    X[out] = rng.random(int(out.sum()))
    U = (U0 + 0.01 * rng.standard_normal((m, k)) / np.sqrt(m)).astype(np.float32)
    Y = (Y0 + 0.05 * rng.standard_normal((k, n))).astype(np.float32)
    labels = (rng.random((n, m // C)) < label_frac).astype(np.uint8)
    return U, Y, np.ascontiguousarray(X, dtype=np.float32), labels


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m,C,k,n,labels_on", [(76800, 1, 10, 64, True), (1000, 1, 3, 5, False),
                                               (2 * 3 * 37, 3, 16, 7, True), (300, 1, 1, 1, True)])
def test_cost_and_gradients_match_the_oracle(m, C, k, n, labels_on):
    p, omega, mu = 0.25, 5e-5, 0.05
    U, Y, X, labels = _case(m, C, k, n, seed=m + k + n)
    if not labels_on:
        labels = None
    W = wo.expand_weights(labels if labels is not None else np.zeros((n, m // C), np.uint8), C, omega)
    F, dU, dY, dmu = wo.window_cost_grad(U, Y, X, W, p, mu)
    win = pg.window.WindowCost(m, C, k, n, p, omega)
    try:
        Ut = torch.from_numpy(U).cuda().requires_grad_()
        Yt = torch.from_numpy(Y).cuda().requires_grad_()
        mut = torch.tensor(mu, dtype=torch.float32, device="cuda").requires_grad_()
        Xt = torch.from_numpy(X).cuda()
        Lt = torch.from_numpy(labels).cuda() if labels is not None else None
        cost = win(Ut, Yt, mut, Xt, Lt)
        (3.0 * cost).backward()
        c = float(cost)
        gU, gY, gmu = Ut.grad.cpu().numpy(), Yt.grad.cpu().numpy(), float(mut.grad)
    finally:
        win.close()
    print(f"m={m} k={k} n={n}: cost {abs(c - F) / F:.1e}, dU {_rel(gU, 3 * dU):.1e}, "
          f"dY {_rel(gY, 3 * dY):.1e}, dmu {abs(gmu - 3 * dmu) / (3 * dmu):.1e}")
    assert abs(c - F) <= COST_RTOL * F
    assert _rel(gU, 3 * dU) <= GRAD_RTOL
    assert _rel(gY, 3 * dY) <= GRAD_RTOL
    assert abs(gmu - 3 * dmu) <= GRAD_RTOL * 3 * dmu
    # element by element, scaled by the largest entry: an error confined to a
    # few rows would pass the norms above but not this
    assert np.max(np.abs(gU - 3 * dU)) <= ELEM_RTOL * np.max(np.abs(3 * dU))
    assert np.max(np.abs(gY - 3 * dY)) <= ELEM_RTOL * np.max(np.abs(3 * dY))


def test_gradients_against_central_differences_of_the_gpu_cost():
    m, C, k, n = 2000, 1, 4, 8
    U, Y, X, labels = _case(m, C, k, n, seed=5)
    win = pg.window.WindowCost(m, C, k, n, 0.5, 0.1)
    rng = np.random.default_rng(6)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        Xt, Lt = dev(X), torch.from_numpy(labels).cuda()
        mu = torch.tensor(0.2, dtype=torch.float32, device="cuda")
        Ut, Yt = dev(U).requires_grad_(), dev(Y).requires_grad_()
        mut = mu.clone().requires_grad_()
        win(Ut, Yt, mut, Xt, Lt).backward()
        for A, G, which in ((U, Ut.grad, 0), (Y, Yt.grad, 1)):
            V = rng.standard_normal(A.shape)
            V /= np.linalg.norm(V)
            h = 1e-2
            args = []
            for s in (1, -1):
                B = A + s * h * V
                args.append(float(win(dev(B), Yt.detach(), mu, Xt, Lt) if which == 0 else
                                  win(Ut.detach(), dev(B), mu, Xt, Lt)))
            fd = (args[0] - args[1]) / (2 * h)
            an = float(np.sum(G.cpu().numpy().astype(np.float64) * V))
            assert fd == pytest.approx(an, rel=2e-2, abs=1e-3 * abs(args[0]))
        h = 1e-2
        fp = float(win(Ut.detach(), Yt.detach(), mu + h, Xt, Lt))
        fm = float(win(Ut.detach(), Yt.detach(), mu - h, Xt, Lt))
        assert (fp - fm) / (2 * h) == pytest.approx(float(mut.grad), rel=2e-2)
    finally:
        win.close()


def test_ustep_matches_the_oracle_and_descends():
    m, C, k, n = 76800, 1, 10, 64
    X, U0, Y0, _ = synth.window_workload()
    rng = np.random.default_rng(7)
    U = synth.random_orthonormal(m, k, rng) * 0.2 + U0 * 0.8
    U = np.linalg.qr(U)[0].astype(np.float32)
    Y = Y0.astype(np.float32)
    p, mu = 0.25, 0.05
    W = np.ones((n, m))
    F, dU, _, _ = wo.window_cost_grad(U, Y, X, W, p, mu)
    t = 1e-3 / float(np.linalg.norm(dU))
    Q = wo.grassmann_window_step(U, dU, t)
    win = pg.window.WindowCost(m, C, k, n, p, 5e-5)
    try:
        Ut = torch.from_numpy(U).cuda()
        dUt = torch.from_numpy(dU.astype(np.float32)).cuda()
        out = torch.empty_like(Ut)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        win.ustep(Ut, dUt, t, out, st)
        torch.cuda.synchronize()
        Qg = out.cpu().numpy()
        status = int(st.item())
    finally:
        win.close()
    assert status == 0
    assert _rel(Qg, Q) <= 1e-5
    np.testing.assert_allclose(Qg.T.astype(np.float64) @ Qg, np.eye(k), atol=1e-5)
    assert wo.window_cost_grad(Qg, Y, X, W, p, mu)[0] < F


def test_argument_checks():
    with pytest.raises(pg.ProstError):
        pg.prost_window_init(100, 3, 4, 8)     # m not a multiple of the channels
    with pytest.raises(pg.ProstError):
        pg.prost_window_init(100, 1, 17, 8)    # k > 16
    with pytest.raises(pg.ProstError):
        pg.prost_window_init(100, 1, 4, 129)   # n > 128


def test_gradient_scale_in_the_kernel():
    """prost_window_eval's gscale multiplies the three gradients inside the
    pass (the C ABI's form of an upstream gradient)."""
    m, C, k, n = 3000, 1, 5, 6
    U, Y, X, labels = _case(m, C, k, n, seed=9)
    w = pg.prost_window_init(m, C, k, n, 0.25, 5e-5)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        Ut, Yt, Xt, Lt = dev(U), dev(Y), dev(X), dev(labels)
        mu = torch.tensor(0.05, dtype=torch.float32, device="cuda")
        g = torch.tensor(-2.5, dtype=torch.float32, device="cuda")
        outs = []
        for gs in (None, g):
            c = torch.empty((), dtype=torch.float32, device="cuda")
            dU, dY, dmu = torch.empty_like(Ut), torch.empty_like(Yt), torch.empty_like(mu)
            pg.prost_window_eval(w, Ut, Yt, Xt, Lt, mu, c, dU, dY, dmu, gscale=gs)
            outs.append((float(c), dU.cpu().numpy(), dY.cpu().numpy(), float(dmu)))
    finally:
        pg.prost_window_destroy(w)
    (c1, u1, y1, m1), (c2, u2, y2, m2) = outs
    assert c1 == c2
    np.testing.assert_allclose(u2, -2.5 * u1, rtol=1e-6, atol=1e-30)
    np.testing.assert_allclose(y2, -2.5 * y1, rtol=1e-6, atol=1e-30)
    assert m2 == pytest.approx(-2.5 * m1, rel=1e-6)
