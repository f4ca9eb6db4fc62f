"""Thin ctypes binding of libffp.so (C ABI in include/ffp.h).

Argument marshalling only: every step of setup, apply, SpMV and the CG solve
runs in the library's CUDA kernels.  PyTorch provides the device memory (the
workspace and vectors) and the current CUDA stream.  There is no CPU fallback:
if libffp.so is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffp.so")
HEADER = os.path.join(_HERE, "..", "include", "ffp.h")

FFP_OK = 0
FFP_ERR_ARG = -1
FFP_ERR_CUDA = -2
FFP_ERR_BREAKDOWN = -3
FFP_ERR_NOT_CONVERGED = -4
FFP_ERR_TIMEOUT = -5
FFP_ERR_UNSUPPORTED = -6
FFP_MAX_NX = 1024

FFP_DIRICHLET, FFP_NEUMANN = 0, 1
FFP_FILTER_ROWSUM, FFP_FILTER_USER = 0, 1
FFP_FP64, FFP_FP32, FFP_BF16 = 0, 1, 2
FFP_PRECOND_NTD, FFP_PRECOND_COMBO = 0, 1
FFP_SCHUR_BETA = 16
PRECISIONS = {"fp64": FFP_FP64, "fp32": FFP_FP32, "bf16": FFP_BF16}
PRECONDS = {"ntd": FFP_PRECOND_NTD, "combo": FFP_PRECOND_COMBO}
SCHURS = {"newton": 0, "beta": FFP_SCHUR_BETA}


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class BC(ctypes.Structure):
    _fields_ = [("face", ctypes.c_ubyte * 6)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("solve_s", ctypes.c_double),
                ("precond_ms", ctypes.c_double), ("ntd_ms", ctypes.c_double),
                ("napply", ctypes.c_int), ("launches", ctypes.c_longlong), ("iters_rec", ctypes.c_int),
                ("spmv_ms", ctypes.c_double), ("lanczos_min", ctypes.c_double),
                ("lanczos_max", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["cond_est"] = (self.lanczos_max / self.lanczos_min) if self.lanczos_min > 0 else float("nan")
        return d


class BatchConfig(ctypes.Structure):
    _fields_ = [("ilu_warps", ctypes.c_int), ("branches", ctypes.c_int), ("ms", ctypes.c_double),
                ("ntd_ms", ctypes.c_double), ("from_cache", ctypes.c_int), ("rhs_per_cta", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FFP_BATCH_MAX_PAIRS = 65535
FFP_NET_PARAMS = 14737
FFP_NET_MAX_NX = 1000


class FFPError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


_lib = None


def declared_functions():
    """Names of the functions include/ffp.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ffp_[a-z_0-9]+)\s*\(", txt)))


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, P = ctypes.c_void_p, ctypes.POINTER
    lib.ffp_workspace_bytes.argtypes = [P(Grid), ctypes.c_int]
    lib.ffp_workspace_bytes.restype = ctypes.c_size_t
    lib.ffp_setup.argtypes = [P(Grid), vp, P(BC), ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                              vp, ctypes.c_size_t, vp, P(vp)]
    lib.ffp_spmv.argtypes = [vp, vp, vp, vp]
    lib.ffp_apply.argtypes = [vp, vp, vp, vp]
    lib.ffp_pcg_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, P(Stats), vp]
    lib.ffp_export.argtypes = [vp] * 11
    lib.ffp_destroy.argtypes = [vp]
    lib.ffp_destroy.restype = None
    lib.ffp_strerror.argtypes = [ctypes.c_int]
    lib.ffp_strerror.restype = ctypes.c_char_p
    lib.ffp_apply_noalloc.argtypes = [vp, vp, vp, vp]
    lib.ffp_debug_stall.argtypes = [vp, ctypes.c_int, ctypes.c_uint]
    lib.ffp_batch_workspace_bytes.argtypes = [ctypes.c_int, P(Grid), ctypes.c_int, ctypes.c_int]
    lib.ffp_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.ffp_batch_setup.argtypes = [ctypes.c_int, P(Grid), P(vp), P(BC), P(vp), ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, vp, P(vp)]
    lib.ffp_batch_tune.argtypes = [vp, ctypes.c_char_p, P(BatchConfig), vp]
    lib.ffp_batch_get_config.argtypes = [vp, P(BatchConfig)]
    lib.ffp_batch_set_config.argtypes = [vp, P(BatchConfig)]
    lib.ffp_batch_info.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_longlong),
                                   P(ctypes.c_longlong)]
    lib.ffp_batch_solve.argtypes = [vp, P(vp), P(vp), ctypes.c_double, ctypes.c_int, P(Stats), vp]
    lib.ffp_batch_destroy.argtypes = [vp]
    lib.ffp_batch_destroy.restype = None
    lib.ffp_net_workspace_bytes.argtypes = [P(Grid), ctypes.c_int, ctypes.c_int]
    lib.ffp_net_workspace_bytes.restype = ctypes.c_size_t
    lib.ffp_net_init.argtypes = [ctypes.c_ulonglong, vp, vp, vp]
    lib.ffp_net_cast.argtypes = [vp, vp, vp]
    lib.ffp_net_forward.argtypes = [P(Grid), ctypes.c_int, vp, vp, vp, vp, ctypes.c_size_t, vp, vp]
    lib.ffp_net_grad.argtypes = [P(Grid), ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_size_t, vp,
                                 P(ctypes.c_double), vp]
    lib.ffp_net_adam.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    lib.ffp_lanczos_scratch_bytes.argtypes = [P(Grid), ctypes.c_int]
    lib.ffp_lanczos_scratch_bytes.restype = ctypes.c_size_t
    lib.ffp_lanczos_ritz.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t,
                                     P(ctypes.c_double), vp, P(ctypes.c_int), vp]
    lib.ffp_filter_target.argtypes = [P(Grid), ctypes.c_int, P(ctypes.c_double), vp,
                                      ctypes.c_double, vp, vp, vp, ctypes.c_size_t, vp]
    for f in (lib.ffp_setup, lib.ffp_spmv, lib.ffp_apply, lib.ffp_pcg_solve, lib.ffp_export,
              lib.ffp_apply_noalloc, lib.ffp_debug_stall, lib.ffp_batch_setup, lib.ffp_batch_tune, lib.ffp_batch_get_config,
              lib.ffp_batch_set_config, lib.ffp_batch_info, lib.ffp_batch_solve, lib.ffp_net_init,
              lib.ffp_net_cast, lib.ffp_net_forward, lib.ffp_net_grad, lib.ffp_net_adam,
              lib.ffp_lanczos_ritz, lib.ffp_filter_target):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def strerror(status):
    try:
        return load().ffp_strerror(int(status)).decode()
    except Exception:  # pragma: no cover - only when the library is missing
        return "unknown"


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _grid(grid, lengths):
    nx, ny, nz = (int(v) for v in grid)
    lx, ly, lz = (float(v) for v in lengths)
    return Grid(nx, ny, nz, lx, ly, lz)


def workspace_bytes(grid, precision="fp64", lengths=(1.0, 1.0, 1.0)):
    g = _grid(grid, lengths)
    return int(load().ffp_workspace_bytes(ctypes.byref(g), PRECISIONS[precision]))


def _dev_vec(x, n, name):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if x.numel() != n or not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous with {n} entries")
    return x


def setup_launches(grid, precond="ntd", user_t=False):
    """Kernels one ffp_setup launches (assembly, filter check, band conversion,
    setup phases, ILU(0) pivot diagonals)."""
    nx, ny, nz = grid
    n = 1 + (1 if user_t else 0) + (4 if precond == "combo" else 2) + (2 if nz > 1 else 1)
    return n + ((ny + nz - 1) if precond == "combo" else 0)


class Preconditioner:
    """Operator A (assembled from kappa) and its preconditioner B on the
    current CUDA device: precond "ntd" (B_NTD, Sec. II) or "combo" (B_c with the
    ILU(0) smoother, Sec. III).  The workspace is a torch uint8 tensor kept by
    this object; the library only points into it."""

    def __init__(self, grid, kappa, bc, precision="fp64", t=None, lengths=(1.0, 1.0, 1.0),
                 stream=None, precond="ntd", workspace=None, schur="newton"):
        """schur: "newton" (X = 2 beta - beta P beta, Sec. II-A as printed) or
        "beta" (X = beta, FFP_SCHUR_BETA)."""
        lib = load()
        self.grid = tuple(int(v) for v in grid)
        self.n = self.grid[0] * self.grid[1] * self.grid[2]
        self.precision = precision
        self.precond = precond
        g = _grid(self.grid, lengths)
        nbytes = lib.ffp_workspace_bytes(ctypes.byref(g), PRECISIONS[precision])
        if nbytes == 0:
            raise FFPError(FFP_ERR_ARG, "ffp_workspace_bytes")
        dev = kappa.device
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        elif not (workspace.is_cuda and workspace.dtype == torch.uint8 and workspace.numel() >= nbytes
                  and workspace.data_ptr() % 256 == 0):
            raise ValueError(f"workspace must be a 256-byte aligned CUDA uint8 tensor of >= {nbytes} bytes")
        self.workspace = workspace
        kappa = _dev_vec(kappa, self.n, "kappa")
        if t is not None:
            t = _dev_vec(t, self.n, "t")
        self._keep = (kappa, t)
        b = BC((ctypes.c_ubyte * 6)(*[int(v) for v in bc]))
        h = ctypes.c_void_p()
        st = lib.ffp_setup(ctypes.byref(g), _ptr(kappa), ctypes.byref(b),
                           FFP_FILTER_USER if t is not None else FFP_FILTER_ROWSUM, _ptr(t),
                           PRECISIONS[precision], PRECONDS[precond] | SCHURS[schur], _ptr(self.workspace),
                           ctypes.c_size_t(nbytes),
                           _stream(stream), ctypes.byref(h))
        if st != FFP_OK:
            raise FFPError(st, "ffp_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().ffp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spmv(self, x, y=None, stream=None):
        x = _dev_vec(x, self.n, "x")
        y = torch.empty_like(x) if y is None else _dev_vec(y, self.n, "y")
        st = load().ffp_spmv(self._h, _ptr(x), _ptr(y), _stream(stream))
        if st != FFP_OK:
            raise FFPError(st, "ffp_spmv")
        return y

    def apply(self, r, z=None, stream=None):
        r = _dev_vec(r, self.n, "r")
        z = torch.empty_like(r) if z is None else _dev_vec(z, self.n, "z")
        st = load().ffp_apply(self._h, _ptr(r), _ptr(z), _stream(stream))
        if st != FFP_OK:
            raise FFPError(st, "ffp_apply")
        return z

    def solve(self, b, x=None, rtol=1e-8, maxit=200, stream=None, check=True):
        """PCG / flexible CG; returns (x, stats dict).  x (if given) is x0 and is
        overwritten with the solution.  The stats are those of ffp_stats: iters,
        iters_rec (first iteration at which the recursive residual met rtol),
        status, rel_res, rel_res_true, solve_s, precond_ms, ntd_ms, napply,
        launches.  A status of FFP_ERR_NOT_CONVERGED means maxit was reached or
        the true residual stopped falling (rtol below the FP64 floor); with
        check=True any status but FFP_OK raises FFPError."""
        b = _dev_vec(b, self.n, "b")
        x = torch.zeros_like(b) if x is None else _dev_vec(x, self.n, "x")
        s = Stats()
        st = load().ffp_pcg_solve(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit),
                                  ctypes.byref(s), _stream(stream))
        if check and st not in (FFP_OK,):
            raise FFPError(st, "ffp_pcg_solve")
        return x, s.as_dict()

    def debug_stall(self, mode, wait_tries=0):
        """Test hook (ffp_debug_stall): mode 1 makes the following applies withhold
        one stage signal so that a bounded wait runs out; mode 0 restores them."""
        st = load().ffp_debug_stall(self._h, int(mode), int(wait_tries))
        if st != FFP_OK:
            raise FFPError(st, "ffp_debug_stall")

    def export(self, names=None, stream=None):
        """Stored operator bands and factors as FP64 device tensors: all of
        d, cx, cy, cz, l3, l2, l1, minv, dinv, or the ones named."""
        allnames = ["d", "cx", "cy", "cz", "l3", "l2", "l1", "minv", "dinv"]
        names = allnames if names is None else list(names)
        out = {k: torch.empty(self.n, dtype=torch.float64, device=self.workspace.device)
               for k in names}
        st = load().ffp_export(self._h, *[_ptr(out.get(k)) for k in allnames], _stream(stream))
        if st != FFP_OK:
            raise FFPError(st, "ffp_export")
        return out


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for k, t in enumerate(tensors):
        arr[k] = None if t is None else t.data_ptr()
    return arr


def batch_workspace_bytes(grids, nrhs, precision="fp32", lengths=None):
    g = (Grid * len(grids))(*[_grid(gr, (lengths[k] if lengths else (1.0, 1.0, 1.0)))
                             for k, gr in enumerate(grids)])
    return int(load().ffp_batch_workspace_bytes(len(grids), g, int(nrhs), PRECISIONS[precision]))


class Batch:
    """Many independent instances (own grid, kappa, boundary conditions and
    preconditioner) with nrhs right-hand sides each, solved together
    (ffp_batch_* in include/ffp.h).  Pairs are numbered i * nrhs + j."""

    def __init__(self, grids, kappas, bcs, nrhs=1, precision="fp32", precond="combo", ts=None,
                 lengths=None, stream=None, workspace=None, schur="newton"):
        lib = load()
        self.grids = [tuple(int(v) for v in g) for g in grids]
        self.count = len(self.grids)
        self.nrhs = int(nrhs)
        self.n = [g[0] * g[1] * g[2] for g in self.grids]
        self.precision, self.precond = precision, precond
        self._g = (Grid * self.count)(*[_grid(gr, (lengths[k] if lengths else (1.0, 1.0, 1.0)))
                                        for k, gr in enumerate(self.grids)])
        nbytes = lib.ffp_batch_workspace_bytes(self.count, self._g, self.nrhs, PRECISIONS[precision])
        if nbytes == 0:
            raise FFPError(FFP_ERR_ARG, "ffp_batch_workspace_bytes")
        kappas = [_dev_vec(k, self.n[i], f"kappa[{i}]") for i, k in enumerate(kappas)]
        dev = kappas[0].device
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        elif not (workspace.is_cuda and workspace.dtype == torch.uint8 and workspace.numel() >= nbytes
                  and workspace.data_ptr() % 256 == 0):
            raise ValueError(f"workspace must be a 256-byte aligned CUDA uint8 tensor of >= {nbytes} bytes")
        self.workspace = workspace
        self.workspace_bytes = nbytes
        if ts is not None:
            ts = [None if t is None else _dev_vec(t, self.n[i], f"t[{i}]") for i, t in enumerate(ts)]
        self._keep = (kappas, ts)
        bca = (BC * self.count)(*[BC((ctypes.c_ubyte * 6)(*[int(v) for v in bc])) for bc in bcs])
        h = ctypes.c_void_p()
        st = lib.ffp_batch_setup(self.count, self._g, _ptr_array(kappas), bca,
                                 _ptr_array(ts) if ts is not None else None, self.nrhs,
                                 PRECISIONS[precision], PRECONDS[precond] | SCHURS[schur],
                                 _ptr(self.workspace),
                                 ctypes.c_size_t(nbytes), _stream(stream), ctypes.byref(h))
        if st != FFP_OK:
            raise FFPError(st, "ffp_batch_setup")
        self._h = h

    @property
    def npairs(self):
        return self.count * self.nrhs

    def pair_size(self, p):
        return self.n[p // self.nrhs]

    def close(self):
        if getattr(self, "_h", None):
            load().ffp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, cache_path=None, stream=None):
        c = BatchConfig()
        st = load().ffp_batch_tune(self._h, cache_path.encode() if cache_path else None,
                                   ctypes.byref(c), _stream(stream))
        if st != FFP_OK:
            raise FFPError(st, "ffp_batch_tune")
        return c.as_dict()

    def config(self):
        c = BatchConfig()
        st = load().ffp_batch_get_config(self._h, ctypes.byref(c))
        if st != FFP_OK:
            raise FFPError(st, "ffp_batch_get_config")
        return c.as_dict()

    def set_config(self, ilu_warps, branches, rhs_per_cta=1):
        c = BatchConfig(int(ilu_warps), int(branches), 0.0, 0.0, 0, int(rhs_per_cta))
        st = load().ffp_batch_set_config(self._h, ctypes.byref(c))
        if st != FFP_OK:
            raise FFPError(st, "ffp_batch_set_config")

    def info(self):
        ng, npair, nl, ns = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        st = load().ffp_batch_info(self._h, ctypes.byref(ng), ctypes.byref(npair), ctypes.byref(nl),
                                   ctypes.byref(ns))
        if st != FFP_OK:
            raise FFPError(st, "ffp_batch_info")
        return {"groups": ng.value, "pairs": npair.value, "launches_per_iter": nl.value,
                "setup_launches": ns.value}

    def solve(self, bs, xs=None, rtol=1e-8, maxit=200, stream=None, check=True):
        """Solve every pair; bs, xs: lists of count * nrhs CUDA float64 tensors
        (xs, if given, hold x0 and receive the solutions).  Returns (xs, stats)."""
        if len(bs) != self.npairs:
            raise ValueError(f"need {self.npairs} right-hand sides")
        bs = [_dev_vec(b, self.pair_size(p), f"b[{p}]") for p, b in enumerate(bs)]
        if xs is None:
            xs = [torch.zeros_like(b) for b in bs]
        else:
            xs = [_dev_vec(x, self.pair_size(p), f"x[{p}]") for p, x in enumerate(xs)]
        stats = (Stats * self.npairs)()
        st = load().ffp_batch_solve(self._h, _ptr_array(bs), _ptr_array(xs), float(rtol), int(maxit),
                                    stats, _stream(stream))
        if check and st != FFP_OK:
            raise FFPError(st, "ffp_batch_solve")
        return xs, [s.as_dict() for s in stats]
