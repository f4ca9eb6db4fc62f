"""FP64 CPU oracle of the learned filter: the 3-D convolutional network that
maps log10(kappa) to a filter vector t > 0, its gradient, the Adam update, the
Lanczos Ritz vectors of B^{-1} A and the training target built from them.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and ``__graft_entry__.smoke``
/ the CPU-baseline leg of ``bench.py``); the CUDA library never calls it.

The paper (Sec. I, the error-propagation argument after Eq. (4)) motivates the
filter: e^{n+1} = (I - B^{-1}A)^{n+1} e^0, a preconditioner with B t = A t
removes the error component along t, and the components that are hardest to
damp lie along the eigenvectors of the smallest eigenvalues of B^{-1}A, so t
should approximate those.  The network, its training and the target are not in
the paper; this module states them plainly:

  features     x0 = log10(kappa) / 3, one channel per cell
  network      four 3x3x3 convolutions with zero padding ("same" size),
               channels 1 -> 16 -> 16 -> 16 -> 1, ReLU after the first three,
               s = output (the log of the filter), t = exp(s)
  conv         y[o, z, y, x] = b[o] + sum_{c, dz, dy, dx} w[o, c, dz, dy, dx]
                               * x[c, z + dz - 1, y + dy - 1, x + dx - 1]
               (cross-correlation, as every deep-learning conv; x = 0 outside)
  loss         L = mean over cells of (s - s*)^2
  target       s* = log t* - mean(log t*), t* = sqrt(sum_k (theta_1/theta_k)
               y_k^2) over the 8 smallest Ritz pairs (theta_k, y_k) of B^{-1}A
               (y_k normalised to max |y_k| = 1), floored at `floor` * max t*
               (the library trains with floor 0.01)
  Adam         Kingma & Ba (2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
               w -= lr * (m / (1-b1^k)) / (sqrt(v / (1-b2^k)) + eps)
  Lanczos      on B^{-1}A, which is self-adjoint in the A-inner product
               <u, v>_A = u^T A v: q_1 = v / ||v||_A, w = B^{-1} A q_j,
               alpha_j = <w, q_j>_A, w -= alpha_j q_j + beta_{j-1} q_{j-1},
               full re-orthogonalisation against every q_i (twice), beta_j =
               ||w||_A with A w recomputed after it, q_{j+1} = w / beta_j; Ritz
               pairs from the tridiagonal (Saad 1996, cited in Sec. I).

BF16 weights: the GPU network stores its weights in BF16 and computes in FP32.
``bf16_round`` gives the value a weight has after that rounding, so the oracle
can run on the very weights the GPU uses.
"""
from __future__ import annotations

import numpy as np

CH = 16
LAYERS = [(1, CH), (CH, CH), (CH, CH), (CH, 1)]   # (in, out) channels per layer


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), via FP32; returns float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(kappa, grid):
    """x0 = log10(kappa) / 3 as a [1, nz, ny, nx] array."""
    nx, ny, nz = grid
    return (np.log10(np.asarray(kappa, dtype=np.float64)) / 3.0).reshape(1, nz, ny, nx)


def init_params(seed=0):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases; w[o, c, dz, dy, dx]."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in LAYERS:
        w = rng.standard_normal((cout, cin, 3, 3, 3)) * np.sqrt(2.0 / (27 * cin))
        params.append((w, np.zeros(cout)))
    return params


def conv3d(x, w, b):
    """Cross-correlation with a 3x3x3 kernel, zero padding, stride 1."""
    cin, nz, ny, nx = x.shape
    cout = w.shape[0]
    xp = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.empty((cout, nz, ny, nx))
    y[:] = b[:, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                y += np.einsum("oc,czyx->ozyx", w[:, :, dz, dy, dx], patch)
    return y


def conv3d_backward(x, w, gy):
    """Gradients of sum(gy * conv3d(x, w, b)) w.r.t. x, w and b."""
    cin, nz, ny, nx = x.shape
    xp = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.empty_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                gw[:, :, dz, dy, dx] = np.einsum("ozyx,czyx->oc", gy, patch)
                gxp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx] += np.einsum(
                    "oc,ozyx->czyx", w[:, :, dz, dy, dx], gy)
    gb = gy.sum(axis=(1, 2, 3))
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gb


def forward(params, x0):
    """Returns s [nz, ny, nx] and the activations (inputs of every layer)."""
    acts = [x0]
    h = x0
    for k, (w, b) in enumerate(params):
        h = conv3d(h, w, b)
        if k < len(params) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h[0], acts


def backward(params, acts, gs):
    """Gradients of sum(gs * s) w.r.t. every (w, b); ReLU derivative 0 at 0."""
    g = gs[None]
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, _ = params[k]
        if k < len(params) - 1:
            g = g * (acts[k + 1] > 0.0)
        gx, gw, gb = conv3d_backward(acts[k], w, g)
        grads[k] = (gw, gb)
        g = gx
    return grads


def loss_and_grad(s, s_target):
    """L = mean (s - s*)^2 and dL/ds."""
    d = s - s_target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state = {"k": step count, "m": [...], "v": [...]}."""
    if not state:
        state["k"] = 0
        state["m"] = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
        state["v"] = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
    state["k"] += 1
    k = state["k"]
    out = []
    for i, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((w, gw), (b, gb))):
            m = state["m"][i][j]
            v = state["v"][i][j]
            m[...] = b1 * m + (1.0 - b1) * g
            v[...] = b2 * v + (1.0 - b2) * g * g
            mh = m / (1.0 - b1 ** k)
            vh = v / (1.0 - b2 ** k)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append((new[0], new[1]))
    return out


def lanczos_ritz(matvec_A, apply_Binv, v0, m):
    """Lanczos on B^{-1}A in the A-inner product with full re-orthogonalisation.
    matvec_A(x) = A x, apply_Binv(r) = B^{-1} r.  Returns (theta ascending,
    Y with the A-normalised Ritz vectors as columns, alpha, beta)."""
    v = np.asarray(v0, dtype=np.float64)
    Av = matvec_A(v)
    nrm = np.sqrt(v @ Av)
    Q, AQ = [v / nrm], [Av / nrm]
    alpha, beta = [], []
    for j in range(m):
        w = apply_Binv(AQ[j])
        alpha.append(float(w @ AQ[j]))
        for _ in range(2):
            for q, aq in zip(Q, AQ):
                w = w - (w @ aq) * q
        Aw = matvec_A(w)  # recomputed: updating it along with w loses accuracy
        bj = np.sqrt(max(float(w @ Aw), 0.0))
        if j == m - 1 or bj <= 1e-14 * abs(alpha[0]):
            break
        beta.append(bj)
        Q.append(w / bj)
        AQ.append(Aw / bj)
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:k - 1], 1) + np.diag(beta[:k - 1], -1)
    theta, S = np.linalg.eigh(T)
    Y = np.stack(Q[:k], axis=1) @ S
    return theta, Y, np.array(alpha), np.array(beta[:k - 1])


def filter_target(theta, Y, nvec=8, floor=1e-2):
    """t* and the mean-free log target s* from the nvec smallest Ritz pairs."""
    nvec = min(nvec, Y.shape[1])
    acc = np.zeros(Y.shape[0])
    for k in range(nvec):
        y = Y[:, k] / np.max(np.abs(Y[:, k]))
        acc += (theta[0] / theta[k]) * y * y
    t = np.sqrt(acc)
    t = np.maximum(t / t.max(), floor)
    s = np.log(t)
    return t, s - s.mean()
