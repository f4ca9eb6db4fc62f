"""ctypes wrapper around the FP64 CPU oracle (``ffp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or calls anything here, and this module never imports the CUDA library.

Every function restates the paper (arXiv 1909.09771) in plain FP64:
  assemble   Sec. I Eq. (2), finite-volume reading (harmonic-mean faces)
  spmv       Sec. II band storage ("only store the bands of A")
  setup      Sec. II-A recurrences for P_i (level 3), T_i (level 2), M_i (level 1)
  apply      Sec. II-B Algorithms 1-7, entry SOLVE(1, N, x, y, n^2, 3)
  pcg        Sec. III PCG conventions (x0 = 0, ||Ax-b||/||b|| < tol, maxit)
  lanczos_extremes   eigenvalues of the Lanczos tridiagonal built from the PCG
                     coefficients (Saad 1996, cited in Sec. I)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libffp_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ffp_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d = ctypes.c_int, ctypes.c_double
            lib.or_assemble.argtypes = [i, i, i, d, d, d, _D, ctypes.c_char_p, _D, _D, _D, _D]
            lib.or_spmv.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D]
            lib.or_setup.argtypes = [i, i, i, _D, _D, _D, _D, _D, i, _D, _D, _D, _D, _D, _D]
            lib.or_apply.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D]
            lib.or_pcg.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, d, i, i,
                                   ctypes.POINTER(i), ctypes.POINTER(d), _D, _D, _D]
            lib.or_ilu0_setup.argtypes = [i, i, i, _D, _D, _D, _D, _D]
            lib.or_ilu0_solve.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D]
            lib.or_combo_apply.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
            for f in (lib.or_assemble, lib.or_spmv, lib.or_setup, lib.or_apply, lib.or_pcg,
                      lib.or_ilu0_setup, lib.or_ilu0_solve, lib.or_combo_apply):
                f.restype = i
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} returned {st}")


def assemble(grid, kappa, bc, lengths=(1.0, 1.0, 1.0)):
    """Bands (d, cx, cy, cz) of the FV operator; grid = (nx, ny, nz); bc = 6 flags
    (x-,x+,y-,y+,z-,z+), 0 = Dirichlet, 1 = Neumann."""
    nx, ny, nz = grid
    n = nx * ny * nz
    kappa = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    assert kappa.size == n
    out = [np.empty(n) for _ in range(4)]
    bcb = bytes(bytearray(int(v) for v in bc))
    _check(_load().or_assemble(nx, ny, nz, *[float(v) for v in lengths], _p(kappa), bcb,
                               *[_p(o) for o in out]), "or_assemble")
    return tuple(out)


def spmv(grid, bands, x):
    nx, ny, nz = grid
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    _check(_load().or_spmv(nx, ny, nz, *[_p(b) for b in bands], _p(x), _p(y)), "or_spmv")
    return y


class Factors:
    """Setup output.  l3 = cz (z-band of A), l2 = Py (y-band of every P_i),
    l1 = To (x-band of every T_k), M = level-1 twisted pivots; Pd/Px and Td are
    the remaining bands of P_i and T_k, kept for the pins."""

    def __init__(self, grid, l3, Pd, Px, Py, Td, To, M):
        self.grid = grid
        self.l3, self.Pd, self.Px, self.Py, self.Td, self.To, self.M = l3, Pd, Px, Py, Td, To, M

    @property
    def l2(self):
        return self.Py

    @property
    def l1(self):
        return self.To


def setup(grid, bands, t=None, schur="newton"):
    """schur: "newton" -- X = 2 beta - beta P beta in the Schur terms (Sec. II-A as
    printed); "beta" -- X = beta (classical filtering)."""
    nx, ny, nz = grid
    n = nx * ny * nz
    d, cx, cy, cz = bands
    outs = [np.empty(n) for _ in range(6)]
    tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    _check(_load().or_setup(nx, ny, nz, _p(d), _p(cx), _p(cy), _p(cz), _p(tt),
                            {"newton": 0, "beta": 1}[schur], *[_p(o) for o in outs]), "or_setup")
    return Factors(grid, cz, *outs)


def apply(f: Factors, r):
    nx, ny, nz = f.grid
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    z = np.empty_like(r)
    _check(_load().or_apply(nx, ny, nz, _p(f.l3), _p(f.l2), _p(f.l1), _p(f.M), _p(r), _p(z)),
           "or_apply")
    return z


def ilu0_setup(grid, bands):
    """Pivots D of ILU(0) of blkD(A) (Sec. III, the smoother of the combination)."""
    nx, ny, nz = grid
    D = np.empty(nx * ny * nz)
    _check(_load().or_ilu0_setup(nx, ny, nz, *[_p(b) for b in bands], _p(D)), "or_ilu0_setup")
    return D


def ilu0_solve(grid, bands, D, r):
    nx, ny, nz = grid
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    z = np.empty_like(r)
    _check(_load().or_ilu0_solve(nx, ny, nz, _p(bands[1]), _p(bands[2]), _p(bands[3]), _p(D),
                                 _p(r), _p(z)), "or_ilu0_solve")
    return z


def combo_apply(grid, bands, f: Factors, D, r):
    """B_c^{-1} r = B_NTD^{-1} r + B_ILU0^{-1} r - B_NTD^{-1} A B_ILU0^{-1} r (Sec. III Eq. (com))."""
    nx, ny, nz = grid
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    z = np.empty_like(r)
    _check(_load().or_combo_apply(nx, ny, nz, *[_p(b) for b in bands], _p(f.l2), _p(f.l1),
                                  _p(f.M), _p(D), _p(r), _p(z)), "or_combo_apply")
    return z


def pcg(grid, bands, f: Factors, b, x0=None, rtol=1e-8, maxit=200, flexible=False, ilu=None):
    """PCG with B_NTD, or with the combination B_c when ilu (pivots of
    ilu0_setup) is given.  Returns dict(x, iters, relres, status, alpha, beta, res)."""
    nx, ny, nz = grid
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    ah, bh, rh = np.zeros(maxit + 1), np.zeros(maxit + 1), np.zeros(maxit + 1)
    st = _load().or_pcg(nx, ny, nz, *[_p(v) for v in bands], _p(f.l2), _p(f.l1), _p(f.M),
                        _p(ilu), _p(b), _p(x), float(rtol), int(maxit), int(bool(flexible)),
                        ctypes.byref(it), ctypes.byref(rr), _p(ah), _p(bh), _p(rh))
    k = it.value
    return dict(x=x, iters=k, relres=rr.value, status=st, alpha=ah[:k].copy(),
                beta=bh[:k].copy(), res=rh[:k].copy())


def lanczos_extremes(alpha, beta):
    """Extreme eigenvalues of the Lanczos tridiagonal of B^{-1}A recovered from
    the CG coefficients (diag 1/a_k + b_k/a_{k-1}, off-diag sqrt(b_k)/a_{k-1}),
    with b_k the coefficient that formed p_k.  Returns (lmin, lmax)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    k = alpha.size
    if k == 0:
        return (np.nan, np.nan)
    diag = np.empty(k)
    off = np.empty(max(k - 1, 0))
    for j in range(k):
        diag[j] = 1.0 / alpha[j]
        if j > 0:
            diag[j] += beta[j] / alpha[j - 1]
            off[j - 1] = np.sqrt(beta[j]) / alpha[j - 1]
    Tm = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(Tm)
    return float(ev[0]), float(ev[-1])
