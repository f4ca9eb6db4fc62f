"""Tolerances the GPU parity tests derive at run time from the oracle.

Two facts about the method fix the tolerances.

1. B^{-1} is entrywise non-negative.  Every T_k is an M-matrix: positive
   pivots and non-positive x-couplings, because the approximate inverse
   2 beta - beta T beta has a positive off-diagonal.  The y- and z-couplings
   l2 and l3 are non-positive, and so the sweeps of Algorithms 2-7 map a
   non-negative right-hand side to a non-negative result.  Hence
   |B^{-1} r| <= B^{-1} |r| entry by entry.  A rounding error made anywhere in
   the apply reaches entry i through the same non-negative operators, so
   s = B^{-1} |r| is the natural per-entry scale: |z_gpu - z_ref|_i <= tol * s_i.
   `apply_scale` checks the non-negativity on the data it is given.

2. The setup is a chain of recurrences.  A backward-stable evaluation of it
   (the GPU's scans, or the oracle's loops) carries a relative error of about
   L * eps in its inputs, L = the longest chain (max(nx, ny, nz)).  Its result
   then differs from the exact one by about cond * L * eps.  `sensitivity`
   measures cond on the oracle itself: it perturbs every operator band by a
   random relative 1e-13, sets up again, and reports the relative change of
   the factors (per entry) and of the apply (per entry of s), each divided by
   1e-13.  Two FP64 evaluations in different rounding orders may then differ
   by 2 * cond * L * eps.  The tests allow 4x that.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as o

EPS = 2.0 ** -53
PERTURB = 1e-13
SAFETY = 4.0


def apply_scale(f, r):
    """s = B^{-1} |r| with the oracle's factors f, and a check that
    B^{-1} |r| >= |B^{-1} r| entry by entry (the non-negativity above)."""
    s = o.apply(f, np.abs(r))
    z = o.apply(f, r)
    assert np.all(s >= np.abs(z) * (1.0 - 1e-10)), "B^{-1} is not entrywise non-negative here"
    return s, z


def sensitivity(grid, bands, f, r, s, seed=99, t=None, schur="newton"):
    """(kappa_factors, amp_apply): the oracle's relative change of the factors
    (l2, l1, 1/M; max per entry) and of the apply (max per entry over s) when
    every band moves by a random relative PERTURB, each divided by PERTURB."""
    rng = np.random.default_rng(seed)
    bp = tuple(b * (1.0 + PERTURB * rng.uniform(-1.0, 1.0, b.size)) for b in bands)
    fp = o.setup(grid, bp, t, schur=schur)

    def rel(a, b):
        return float(np.max(np.abs(a - b) / (np.abs(b) + 1e-300)))

    kf = max(rel(fp.Py, f.Py), rel(fp.To, f.To), rel(1.0 / fp.M, 1.0 / f.M)) / PERTURB
    za = o.apply(f, r)
    zp = o.apply(fp, r)
    amp = float(np.max(np.abs(zp - za) / s)) / PERTURB
    return kf, amp


def chain(grid):
    return float(max(grid))


def factor_tol(grid, kf):
    """Per-entry relative tolerance of the FP64 setup factors, GPU vs oracle."""
    return max(1e-13, 2.0 * SAFETY * chain(grid) * EPS * max(kf, 1.0))


def e2e_tol(grid, amp, apply_tol=1e-12):
    """Per-entry tolerance (in units of s = B^{-1}|r|) of the FP64 setup + apply,
    GPU vs oracle: the apply's own rounding plus the setup's, carried through
    the apply."""
    return apply_tol + 2.0 * SAFETY * chain(grid) * EPS * max(amp, 1.0)


def per_entry_ok(z, zr, s, tol):
    """max_i |z_i - zr_i| / s_i <= tol; returns (ok, worst ratio)."""
    worst = float(np.max(np.abs(z - zr) / s))
    return worst <= tol, worst
