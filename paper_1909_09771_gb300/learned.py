"""Learned filter vector t for the nested filtering preconditioner.

Sec. I of the paper: with B t = A t the error component along t is removed,
and the slowest components lie along the eigenvectors of the smallest
eigenvalues of B^{-1}A, so t should approximate them.  This module trains the
library's convolutional network (include/ffp.h, "Learned filter") to predict
such a t from log10(kappa):
  1. targets: for each training instance, Lanczos Ritz vectors of
     B_rowsum^{-1} A (ffp_lanczos_ritz) -> t*, s* = log t* - mean
     (ffp_filter_target);
  2. training: minibatches of (kappa, s*) -> ffp_net_grad -> ffp_net_adam;
  3. use: ffp_net_forward gives t, passed to ffp_setup as FFP_FILTER_USER.
Host orchestration only: every arithmetic step is a call into libffp.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import ffp
from . import inputs as I


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class FilterNet:
    """Network parameters (FP32 master copy, BF16 copy, Adam moments) on one device."""

    def __init__(self, seed=0, device="cuda", stream=None):
        lib = ffp.load()
        self.device = torch.device(device)
        P = ffp.FFP_NET_PARAMS
        self.params = torch.zeros(P, dtype=torch.float32, device=self.device)
        self.wbf16 = torch.zeros(P, dtype=torch.int16, device=self.device)
        self.m = torch.zeros(P, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(P, dtype=torch.float32, device=self.device)
        self.step = 0
        st = lib.ffp_net_init(ctypes.c_ulonglong(seed), _p(self.params), _p(self.wbf16),
                              ffp._stream(stream))
        if st != ffp.FFP_OK:
            raise ffp.FFPError(st, "ffp_net_init")
        self._ws = {}

    def load(self, params, stream=None):
        """Set the FP32 parameters (and their BF16 copy) from an array."""
        self.params.copy_(torch.as_tensor(np.asarray(params, dtype=np.float32)))
        st = ffp.load().ffp_net_cast(_p(self.params), _p(self.wbf16), ffp._stream(stream))
        if st != ffp.FFP_OK:
            raise ffp.FFPError(st, "ffp_net_cast")

    def _workspace(self, grid, batch, train):
        key = (tuple(grid), batch, train)
        if key not in self._ws:
            g = ffp._grid(grid, (1.0, 1.0, 1.0))
            nb = ffp.load().ffp_net_workspace_bytes(ctypes.byref(g), batch, train)
            if nb == 0:
                raise ffp.FFPError(ffp.FFP_ERR_ARG, "ffp_net_workspace_bytes")
            self._ws = {key: torch.empty(nb, dtype=torch.uint8, device=self.device)}
        return self._ws[key]

    def forward(self, grid, kappa, batch=1, t=None, stream=None):
        """t = exp(s) for `batch` instances (kappa FP64 [batch * N] device)."""
        n = int(np.prod(grid))
        ws = self._workspace(grid, batch, 0)
        t = torch.empty(batch * n, dtype=torch.float64, device=self.device) if t is None else t
        g = ffp._grid(grid, (1.0, 1.0, 1.0))
        st = ffp.load().ffp_net_forward(ctypes.byref(g), batch, _p(kappa), _p(self.params),
                                        _p(self.wbf16), _p(ws), ctypes.c_size_t(ws.numel()), _p(t),
                                        ffp._stream(stream))
        if st != ffp.FFP_OK:
            raise ffp.FFPError(st, "ffp_net_forward")
        return t

    def grad(self, grid, kappa, s_target, batch=1, grad=None, stream=None, want_loss=True):
        ws = self._workspace(grid, batch, 1)
        grad = torch.empty(ffp.FFP_NET_PARAMS, dtype=torch.float32, device=self.device) \
            if grad is None else grad
        g = ffp._grid(grid, (1.0, 1.0, 1.0))
        loss = ctypes.c_double(0.0)
        st = ffp.load().ffp_net_grad(ctypes.byref(g), batch, _p(kappa), _p(s_target),
                                     _p(self.params), _p(self.wbf16), _p(ws),
                                     ctypes.c_size_t(ws.numel()), _p(grad),
                                     ctypes.byref(loss) if want_loss else None, ffp._stream(stream))
        if st != ffp.FFP_OK:
            raise ffp.FFPError(st, "ffp_net_grad")
        return grad, (loss.value if want_loss else None)

    def adam(self, grad, lr=1e-3, stream=None):
        self.step += 1
        st = ffp.load().ffp_net_adam(_p(self.params), _p(self.wbf16), _p(self.m), _p(self.v),
                                     _p(grad), self.step, float(lr), ffp._stream(stream))
        if st != ffp.FFP_OK:
            raise ffp.FFPError(st, "ffp_net_adam")


def lanczos_ritz(P, m=40, nvec=8, seed=0, stream=None):
    """Ritz values (numpy, ascending) and the nvec smallest A-normalised Ritz
    vectors (device FP64 [nvec][N]) of B_NTD^{-1}A for Preconditioner P."""
    lib = ffp.load()
    n = P.n
    g = ffp._grid(P.grid, (1.0, 1.0, 1.0))
    nb = lib.ffp_lanczos_scratch_bytes(ctypes.byref(g), m)
    scratch = torch.empty(nb, dtype=torch.uint8, device=P.workspace.device)
    v0 = torch.as_tensor(I.lanczos_start(n, seed), device=P.workspace.device)
    Y = torch.empty(max(nvec, 1) * n, dtype=torch.float64, device=P.workspace.device)
    theta = (ctypes.c_double * m)()
    steps = ctypes.c_int(0)
    st = lib.ffp_lanczos_ritz(P._h, _p(v0), m, nvec, _p(scratch), ctypes.c_size_t(nb), theta, _p(Y),
                              ctypes.byref(steps), ffp._stream(stream))
    if st != ffp.FFP_OK:
        raise ffp.FFPError(st, "ffp_lanczos_ritz")
    return np.array(theta[:steps.value]), Y.view(nvec, n) if nvec > 0 else None, scratch


FLOOR = 0.003  # target floor (relative to max t*) of the trained network


def filter_target(grid, theta, Y, nvec=8, floor=FLOOR, scratch=None, stream=None):
    """(t* FP64, s* FP32) device vectors from the Ritz pairs."""
    lib = ffp.load()
    n = int(np.prod(grid))
    g = ffp._grid(grid, (1.0, 1.0, 1.0))
    nb = lib.ffp_lanczos_scratch_bytes(ctypes.byref(g), 1)
    if scratch is None or scratch.numel() < nb:
        scratch = torch.empty(nb, dtype=torch.uint8, device=Y.device)
    t = torch.empty(n, dtype=torch.float64, device=Y.device)
    s = torch.empty(n, dtype=torch.float32, device=Y.device)
    th = (ctypes.c_double * nvec)(*[float(v) for v in theta[:nvec]])
    st = lib.ffp_filter_target(ctypes.byref(g), nvec, th, _p(Y), float(floor), _p(t), _p(s),
                               _p(scratch), ctypes.c_size_t(scratch.numel()), ffp._stream(stream))
    if st != ffp.FFP_OK:
        raise ffp.FFPError(st, "ffp_filter_target")
    return t, s


def make_targets(instances, m=40, nvec=8, floor=FLOOR, precision="fp32", device="cuda",
                 max_seconds=None):
    """Per instance: kappa (device FP64) and the target s* (device FP32); stops
    early once max_seconds have passed."""
    import time
    t0 = time.time()
    kappas, targets = [], []
    for k, w in enumerate(instances):
        if max_seconds is not None and time.time() - t0 > max_seconds:
            break
        kap = torch.as_tensor(w["kappa"], device=device)
        P = ffp.Preconditioner(w["grid"], kap, w["bc"], precision, precond="ntd")
        theta, Y, scratch = lanczos_ritz(P, m=m, nvec=nvec, seed=k)
        _, s = filter_target(w["grid"], theta, Y, nvec=nvec, floor=floor, scratch=scratch)
        P.close()
        kappas.append(kap)
        targets.append(s)
    return kappas, targets


def train(net, grid, kappas, targets, epochs=4, batch=8, lr=1e-3, seed=0, log=None):
    """Adam on minibatches of `batch` instances; returns the mean loss per epoch."""
    n = int(np.prod(grid))
    dev = net.device
    kb = torch.empty(batch * n, dtype=torch.float64, device=dev)
    sb = torch.empty(batch * n, dtype=torch.float32, device=dev)
    g = torch.empty(ffp.FFP_NET_PARAMS, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(kappas))
        losses = []
        for b0 in range(0, len(order) - batch + 1, batch):
            for j, i in enumerate(order[b0:b0 + batch]):
                kb[j * n:(j + 1) * n].copy_(kappas[i])
                sb[j * n:(j + 1) * n].copy_(targets[i])
            _, loss = net.grad(grid, kb, sb, batch=batch, grad=g)
            net.adam(g, lr=lr)
            losses.append(loss)
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


# The trained network (target floor 0.003): it lowers the Lanczos estimate of
# cond(B^{-1}A) of plain B_NTD by two to three orders of magnitude on 64^3 GRF
# instances and saves 24-32 % of the B_c iterations on 350^3 instances of contrast
# 10^6; the floor-0.1 network is kept beside it for comparison.
WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "learned_filter_weights.txt")
WEIGHTS_FLOOR01 = __import__("os").path.join(__import__("os").path.dirname(__file__),
                                             "learned_filter_weights_floor01.txt")


def save_weights(net, path):
    np.savetxt(path, net.params.detach().cpu().numpy().astype(np.float64), fmt="%.9e")


def load_weights(path=WEIGHTS, seed=0, device="cuda"):
    net = FilterNet(seed=seed, device=device)
    net.load(np.loadtxt(path))
    return net


def predict_filter(net, w, device="cuda"):
    """t for one instance (dict with grid and kappa), device FP64."""
    kap = torch.as_tensor(w["kappa"], device=device)
    return net.forward(w["grid"], kap, batch=1)


# Floating-point operations of the network per cell: useful ones (the 3x3x3
# convolutions of 1 -> 16 -> 16 -> 16 -> 1 channels) and the ones the tensor
# cores issue (every layer as 16 x 16 channels, the weight gradient with its
# 128-row M of which 16 rows are used, plus the bias-gradient MMA), per cell
# of the padded grid.
USEFUL_FWD = 2 * 27 * (1 * 16 + 16 * 16 + 16 * 16 + 16 * 1)
USEFUL_BWD = 2 * 27 * (1 * 16 + 16 * 16 + 16 * 16) + USEFUL_FWD  # data gradients of layers 3-1, weight gradients
ISSUED_FWD = 4 * 27 * 2 * 16 * 16
ISSUED_BWD = 3 * 27 * 2 * 16 * 16 + 4 * 28 * 2 * 128 * 16


def bench(n=256, train_n=64, train_batch=8, reps=10):
    """CUDA-event times of one forward pass at n^3 and one gradient (forward,
    loss, backward) of a batch of train_n^3 instances, with the useful and
    issued tensor-core TFLOP/s they reach."""
    import json as _json
    import os
    dev = torch.device("cuda")
    net = FilterNet(seed=0)
    out = {}
    peak = None
    pk = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            peak = _json.load(fh).get("bf16_tflops")
    for label, grid, batch in (("forward", (n, n, n), 1), ("gradient", (train_n,) * 3, train_batch)):
        cells = int(np.prod(grid)) * batch
        padded = int(np.prod([v + 2 for v in grid])) * batch
        kap = torch.as_tensor(np.concatenate([I.workload_grf(seed=k, n=grid[0], exponent=2.0)["kappa"]
                                              for k in range(batch)]), device=dev)
        if label == "forward":
            t = torch.empty(cells, dtype=torch.float64, device=dev)
            run = lambda: net.forward(grid, kap, batch=batch, t=t)
            useful, issued = USEFUL_FWD * cells, ISSUED_FWD * padded
        else:
            st = torch.zeros(cells, dtype=torch.float32, device=dev)
            gbuf = torch.empty(ffp.FFP_NET_PARAMS, dtype=torch.float32, device=dev)
            run = lambda: net.grad(grid, kap, st, batch=batch, grad=gbuf, want_loss=False)
            useful, issued = (USEFUL_FWD + USEFUL_BWD) * cells, (ISSUED_FWD + ISSUED_BWD) * padded
        for _ in range(3):
            run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[label] = {"grid": list(grid), "batch": batch, "ms": ms, "cells_per_s": cells / ms * 1e3,
                      "useful_tflops": useful / ms / 1e9, "issued_tflops": issued / ms / 1e9,
                      "issued_frac_of_bf16_peak": (issued / ms / 1e9 / peak) if peak else None}
    out["peak_bf16_tflops"] = peak
    out["note"] = ("whole calls: guard zeroing, weight images, features, the four convolutions (and "
                   "the backward pass), the head, and the call's final synchronisation")
    return out


def _main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="train / evaluate the learned filter network")
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--count", type=int, default=2000)
    tr.add_argument("--n", type=int, default=64)
    tr.add_argument("--epochs", type=int, default=6)
    tr.add_argument("--batch", type=int, default=8)
    tr.add_argument("--lr", type=float, default=2e-3)
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--log", default=None)
    tr.add_argument("--max-target-seconds", type=float, default=None)
    tr.add_argument("--floor", type=float, default=FLOOR,
                    help="target floor relative to max t*")
    tr.add_argument("--exponent", type=float, default=2.0,
                    help="training kappa = 10^(exponent g), contrast 10^(2 exponent)")
    ev = sub.add_parser("eval")
    ev.add_argument("--weights", default=WEIGHTS)
    ev.add_argument("--n", type=int, default=64)
    ev.add_argument("--exponent", type=float, default=2.0)
    ev.add_argument("--seeds", default="0,1")
    ev.add_argument("--precision", default="fp32")
    ev.add_argument("--precond", default="combo,ntd",
                    help="preconditioners to compare the filters with (combo = B_c, ntd = B_NTD)")
    ev.add_argument("--maxit", type=int, default=1000)
    ev.add_argument("--out", default=None)
    bn = sub.add_parser("bench", help="time the network's forward pass and gradient (CUDA events)")
    bn.add_argument("--n", type=int, default=256, help="forward pass on one n^3 instance")
    bn.add_argument("--train-n", type=int, default=64)
    bn.add_argument("--train-batch", type=int, default=8)
    bn.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    ffp.load()
    dev = torch.device("cuda")
    if a.cmd == "bench":
        print(json.dumps(bench(a.n, a.train_n, a.train_batch, a.reps)))
        return
    if a.cmd == "train":
        t0 = time.time()
        insts = I.workload_learned_train(count=a.count, n=a.n, exponent=a.exponent)
        kappas, targets = make_targets(insts, floor=a.floor, max_seconds=a.max_target_seconds)
        t_targets = time.time() - t0
        print(f"targets: {len(kappas)} instances in {t_targets:.1f} s", flush=True)
        net = FilterNet(seed=0)
        t0 = time.time()
        hist = train(net, (a.n,) * 3, kappas, targets, epochs=a.epochs, batch=a.batch, lr=a.lr,
                     log=print)
        t_train = time.time() - t0
        save_weights(net, a.out)
        rep = {"count": len(kappas), "requested": a.count, "n": a.n, "epochs": a.epochs, "floor": a.floor,
               "exponent": a.exponent,
               "batch": a.batch, "lr": a.lr,
               "targets_s": t_targets, "train_s": t_train, "loss": hist}
        print(json.dumps(rep))
        if a.log:
            with open(a.log, "w") as fh:
                json.dump(rep, fh)
    else:
        net = load_weights(a.weights)
        res = []
        for sd in [int(v) for v in a.seeds.split(",")]:
            w = I.workload_grf(seed=sd, n=a.n, exponent=a.exponent)
            kap = torch.as_tensor(w["kappa"], device=dev)
            b = torch.as_tensor(w["b"], device=dev)
            row = {"seed": sd}
            torch.cuda.synchronize()
            t0 = time.time()
            t = predict_filter(net, w)
            torch.cuda.synchronize()
            row["infer_s"] = time.time() - t0
            for pc in a.precond.split(","):
                for name, tt in (("rowsum", None), ("learned", t)):
                    t0 = time.time()
                    P = ffp.Preconditioner(w["grid"], kap, w["bc"], a.precision, t=tt, precond=pc)
                    x, st = P.solve(b, rtol=1e-8, maxit=a.maxit, check=False)
                    torch.cuda.synchronize()
                    # cond_est: Lanczos estimate of cond(B^{-1} A) from the CG coefficients
                    row[f"{pc}_{name}"] = {"iters": st["iters"], "status": st["status"],
                                           "rel_res_true": st["rel_res_true"],
                                           "lanczos_min": st["lanczos_min"],
                                           "lanczos_max": st["lanczos_max"],
                                           "cond_est": st["cond_est"], "s": time.time() - t0}
                    P.close()
            res.append(row)
            print(json.dumps(row), flush=True)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh)


if __name__ == "__main__":
    _main()
