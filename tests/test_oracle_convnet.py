"""Pins of the learned-filter oracle (oracle/convnet.py) to things other than
itself: the convolution against scipy.ndimage.correlate, the gradients against
central finite differences, Adam's first step against its closed form, BF16
rounding against hand-computed values, and the Lanczos Ritz pairs against the
dense generalized eigenproblem of (A, B) on small grids."""
import numpy as np
import pytest
from scipy import linalg, ndimage

from oracle import convnet as C
from oracle import oracle as o
from paper_1909_09771_gb300 import inputs as I


def test_bf16_round_values():
    e = 2.0 ** -8
    vals = np.array([1.0, 1.0 + e, 1.0 + 3 * e, 1.0 + 2 * e, -2.5, 3.0e-39, 1.0 + 1.01 * e])
    want = np.array([1.0, 1.0, 1.0 + 4 * e, 1.0 + 2 * e, -2.5, 0.0, 1.0 + 2 * e])
    got = C.bf16_round(vals)
    assert got[:5].tolist() == want[:5].tolist()
    assert abs(got[5]) < 1e-38            # FP32 subnormal rounds to a BF16 subnormal near 0
    assert got[6] == want[6]


def test_conv3d_equals_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    y = C.conv3d(x, w, b)
    for oc in range(2):
        ref = b[oc] + sum(ndimage.correlate(x[c], w[oc, c], mode="constant", cval=0.0)
                          for c in range(3))
        assert np.max(np.abs(y[oc] - ref)) <= 1e-12 * np.max(np.abs(ref))


def _loss(params, x0, st):
    s, _ = C.forward(params, x0)
    return C.loss_and_grad(s, st)[0]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    grid = (5, 4, 3)
    x0 = rng.standard_normal((1, 3, 4, 5))
    params = C.init_params(seed=2)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    st = rng.standard_normal((3, 4, 5))
    s, acts = C.forward(params, x0)
    _, gs = C.loss_and_grad(s, st)
    grads = C.backward(params, acts, gs)
    h = 1e-6
    for layer in range(4):
        w, b = params[layer]
        for _ in range(6):
            idx = tuple(rng.integers(0, n) for n in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = [p if k != layer else (wp, b) for k, p in enumerate(params)]
            pm = [p if k != layer else (wm, b) for k, p in enumerate(params)]
            fd = (_loss(pp, x0, st) - _loss(pm, x0, st)) / (2 * h)
            assert abs(fd - grads[layer][0][idx]) <= 1e-6 * max(1.0, abs(fd))
        j = int(rng.integers(0, b.size))
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        pp = [p if k != layer else (w, bp) for k, p in enumerate(params)]
        pm = [p if k != layer else (w, bm) for k, p in enumerate(params)]
        fd = (_loss(pp, x0, st) - _loss(pm, x0, st)) / (2 * h)
        assert abs(fd - grads[layer][1][j]) <= 1e-6 * max(1.0, abs(fd))


def test_conv_input_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 4, 3))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = np.zeros(3)
    gy = rng.standard_normal((3, 3, 4, 3))
    gx, _, gb = C.conv3d_backward(x, w, gy)
    assert np.allclose(gb, gy.sum(axis=(1, 2, 3)))
    h = 1e-6
    for _ in range(8):
        idx = tuple(rng.integers(0, n) for n in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (np.sum(gy * C.conv3d(xp, w, b)) - np.sum(gy * C.conv3d(xm, w, b))) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    w = np.array([0.5, -1.0, 2.0])
    g = np.array([0.3, -0.02, 4.0])
    params = [(w.reshape(3, 1, 1, 1, 1) * 0 + w.reshape(3, 1, 1, 1, 1), np.zeros(3))]
    grads = [(g.reshape(3, 1, 1, 1, 1), np.zeros(3))]
    state = {}
    out = C.adam_step(params, grads, state, lr=0.01)
    # first step: m_hat = g, v_hat = g^2  =>  w -= lr * g / (|g| + eps)
    want = w - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(out[0][0].ravel(), want, rtol=0, atol=1e-15)
    assert np.allclose(out[0][1], 0.0)      # zero gradient leaves the bias in place
    assert state["k"] == 1


def _dense_pencil(grid, bands, f):
    n = int(np.prod(grid))
    eye = np.eye(n)
    A = np.stack([o.spmv(grid, bands, eye[:, j]) for j in range(n)], axis=1)
    Binv = np.stack([o.apply(f, eye[:, j]) for j in range(n)], axis=1)
    return A, Binv


@pytest.mark.parametrize("grid", [(5, 4, 3), (6, 5, 4)])
def test_lanczos_ritz_pairs_match_dense_pencil(grid):
    w = I.random_small(grid, 21, contrast_exp=2)
    bands = o.assemble(grid, w["kappa"], w["bc"])
    f = o.setup(grid, bands)
    A, Binv = _dense_pencil(grid, bands, f)
    Bmat = np.linalg.inv(0.5 * (Binv + Binv.T))
    ev, V = linalg.eigh(A, 0.5 * (Bmat + Bmat.T))
    n = A.shape[0]
    theta, Y, _, _ = C.lanczos_ritz(lambda x: A @ x, lambda r: Binv @ r,
                                    np.random.default_rng(5).standard_normal(n), m=n)
    # a full Lanczos run reproduces the extreme eigenvalues of B^{-1}A
    assert abs(theta[0] - ev[0]) <= 1e-8 * ev[-1]
    assert abs(theta[-1] - ev[-1]) <= 1e-8 * ev[-1]
    # and the eigenvector of the smallest one (A-inner product cosine)
    y, v = Y[:, 0], V[:, 0]
    cos = abs(y @ A @ v) / np.sqrt((y @ A @ y) * (v @ A @ v))
    assert cos >= 1 - 1e-8
    # Ritz vectors are A-orthonormal
    G = Y.T @ A @ Y
    assert np.max(np.abs(G - np.eye(G.shape[0]))) <= 1e-8


def test_filter_target_is_positive_floored_and_mean_free():
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((50, 8))
    theta = np.sort(rng.uniform(0.1, 1.0, 8))
    t, s = C.filter_target(theta, Y, floor=0.05)
    assert np.all(t >= 0.05) and t.max() == 1.0
    assert abs(s.mean()) <= 1e-14
    assert np.allclose(np.exp(s) / np.exp(s).max(), t)


def test_filter_target_golden_two_ritz_pairs():
    """The target against a hand-derived fixture (tests/golden/filter_target_two_ritz.txt):
    two Ritz pairs, per-vector max-normalisation, weights theta_0 / theta_k,
    the square root of the weighted sum, scaling to max 1, the floor and the
    mean-free log.  Inverting the weights, dropping the normalisation or the
    square root, or flooring before scaling each changes the values."""
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "filter_target_two_ritz.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    theta = np.array(rows[0])
    Y = np.array(rows[1:4])
    for floor, (t_exp, s_exp) in ((0.1, rows[4:6]), (0.6, rows[6:8])):
        t, s = C.filter_target(theta, Y, nvec=2, floor=floor)
        np.testing.assert_allclose(t, t_exp, rtol=1e-15)
        np.testing.assert_allclose(s, s_exp, rtol=1e-14)
