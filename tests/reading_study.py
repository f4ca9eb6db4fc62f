"""Dense study of the readings of Sec. II-A (small grids only).

A dense, independent construction of the nested twisted preconditioner
B = (B_P + L3) B_P^{-1} (B_P + U3), B_P = (T + L2) T^{-1} (T + U2) per plane,
with a choice, at each of levels 3 and 2, of the approximate inverse X of
the eliminated block that enters the Schur term C X C:
  "newton"  X = 2 beta - beta P beta, beta = diag((P^{-1} w) ./ w)  (the
            paper's formula, Sec. II-A)
  "beta"    X = beta (classical filtering: X w = P^{-1} w, nothing more)
  "exact"   X = P^{-1} (dense; no approximation at that level)
and, at level 3, of the inverse inside beta-hat:
  "nested"  the nested solve B_P^{-1} of the previous plane (reading R1, the
            library's and the oracle's)
  "exact"   the exact inverse of the previous approximated plane P_{i-1}.
The filter vector is t = 1 (rowsum) unless given; the twist block is
m = floor((n-1)/2) at both levels, both halves eliminated towards it, and the
twist block takes both corrections.

It shares no code with the oracle or the CUDA library; the as-written
variant ("newton", "newton", "nested") reproduces the oracle's apply, which
tests/test_reading_study.py checks.  Run as a script it prints, for the
paper's three test matrices and two of this repository's workloads, the
extreme eigenvalues of B^{-1} A, the most negative eigenvalue of the X
matrices relative to their largest, and the CG iterations of B_NTD and of the
combination with ILU(0) (Sec. III Eq. (com)) to 1e-8:

    python -m tests.reading_study [n ...]     (default 8 12)
"""
from __future__ import annotations

import sys

import numpy as np
import scipy.linalg as sla

from tests import dense_ref as D


def _twisted_chain(nb, blocks, coupling, approx_inv, make_x):
    """Twisted Schur recurrence over nb diagonal blocks (dense).  blocks[q]:
    the diagonal block q; coupling[q]: diagonal (vector) coupling blocks q and
    q+1; approx_inv(Q, w): the vector Q^{-1} w used by beta; make_x(Q, beta):
    the approximate inverse X.  Returns the new diagonal blocks and the X
    matrices formed."""
    m = (nb - 1) // 2
    out = [None] * nb
    xs = []

    def schur(prev, c, blk_t):
        w = c * blk_t
        v = approx_inv(prev, w)
        beta = v / w
        X = make_x(prev, beta)
        xs.append(X)
        return (c[:, None] * X) * c[None, :]

    out[0] = blocks[0].copy()
    for q in range(1, m):
        out[q] = blocks[q] - schur(out[q - 1], coupling[q - 1], 1.0)
    if nb - 1 > m:
        out[nb - 1] = blocks[nb - 1].copy()
        for q in range(nb - 2, m, -1):
            out[q] = blocks[q] - schur(out[q + 1], coupling[q], 1.0)
    corr = np.zeros_like(blocks[m])
    if m > 0:
        corr += schur(out[m - 1], coupling[m - 1], 1.0)
    if m < nb - 1:
        corr += schur(out[m + 1], coupling[m], 1.0)
    out[m] = blocks[m] - corr if (m > 0 or m < nb - 1) else blocks[m].copy()
    if nb == 1:
        out[0] = blocks[0].copy()
    return out, xs


def _xmaker(kind):
    if kind == "newton":
        return lambda P, beta: 2.0 * np.diag(beta) - (beta[:, None] * P) * beta[None, :]
    if kind == "beta":
        return lambda P, beta: np.diag(beta)
    if kind == "exact":
        return lambda P, beta: np.linalg.inv(P)
    raise ValueError(kind)


def plane_bp(P, nx, ny, x2="newton"):
    """B_P of one plane matrix P (dense nxy x nxy) and the level-2 X matrices."""
    blocks = [P[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx] for k in range(ny)]
    coup = [np.diag(P[k * nx:(k + 1) * nx, (k + 1) * nx:(k + 2) * nx]).copy() for k in range(ny - 1)]
    T, xs = _twisted_chain(ny, blocks, coup, lambda Q, w: np.linalg.solve(Q, w), _xmaker(x2))
    Td = sla.block_diag(*T)
    py = np.concatenate([c for c in coup] + [np.zeros(nx)]) if ny > 1 else np.zeros(nx)
    L2 = D.twisted_lower(ny, nx, py)
    BP = (Td + L2) @ np.linalg.solve(Td, Td + L2.T)
    return BP, xs


def dense_ntd(grid, bands, x3="newton", x2="newton", beta3="nested"):
    """Dense B_NTD for the given readings; returns (B, X3 list, X2 list)."""
    nx, ny, nz = grid
    nxy = nx * ny
    A = D.dense_A(grid, bands)
    blocks = [A[i * nxy:(i + 1) * nxy, i * nxy:(i + 1) * nxy] for i in range(nz)]
    coup = [np.diag(A[i * nxy:(i + 1) * nxy, (i + 1) * nxy:(i + 2) * nxy]).copy() for i in range(nz - 1)]
    x2s = []

    def inv3(P, w):
        if beta3 == "exact":
            return np.linalg.solve(P, w)
        BP, _ = plane_bp(P, nx, ny, x2)
        return np.linalg.solve(BP, w)

    P, x3s = _twisted_chain(nz, blocks, coup, inv3, _xmaker(x3))
    BPs = []
    for Pi in P:
        if x3 == "exact":
            BPs.append(Pi)           # dense Schur complements: no level-2 structure left
        else:
            BP, xs = plane_bp(Pi, nx, ny, x2)
            BPs.append(BP)
            x2s.extend(xs)
    BP = sla.block_diag(*BPs)
    cz = np.concatenate(coup + [np.zeros(nxy)]) if nz > 1 else np.zeros(nxy)
    L3 = D.twisted_lower(nz, nxy, cz)
    B = (BP + L3) @ np.linalg.solve(BP, BP + L3.T)
    return 0.5 * (B + B.T), x3s, x2s


def indefiniteness(xs):
    """Most negative eigenvalue of the symmetric X matrices relative to their
    largest, over the list (0 if all are positive semidefinite)."""
    worst = 0.0
    for X in xs:
        ev = np.linalg.eigvalsh(0.5 * (X + X.T))
        worst = min(worst, ev[0] / max(abs(ev[-1]), 1e-300))
    return worst


def cg_iters(A, apply_inv, b, rtol=1e-8, maxit=2000, flexible=False):
    """(flexible) preconditioned CG from x0 = 0 to ||b - A x|| / ||b|| < rtol."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    z = apply_inv(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r_old = r
        r = r - alpha * q
        if np.linalg.norm(r) / bn < rtol:
            return it
        z = apply_inv(r)
        rz_new = r @ z
        beta = (rz_new - (z @ r_old if flexible else 0.0)) / rz
        rz = rz_new
        p = z + beta * p
    return maxit


def ilu0_dense(grid, A):
    """ILU(0) of blkD(A) (Sec. III): block-diagonal split at M = floor(N/2),
    no fill outside the pattern of A; returns a function r -> B_ILU0^{-1} r."""
    n = A.shape[0]
    M = n // 2
    Ab = A.copy()
    Ab[:M, M:] = 0.0
    Ab[M:, :M] = 0.0
    pattern = Ab != 0.0
    LU = Ab.copy()
    for i in range(1, n):
        for k in range(i):
            if pattern[i, k] and LU[k, k] != 0.0:
                LU[i, k] /= LU[k, k]
                row = pattern[i, k + 1:]
                LU[i, k + 1:][row] -= LU[i, k] * LU[k, k + 1:][row]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    return lambda r: sla.solve_triangular(U, sla.solve_triangular(L, r, lower=True, unit_diagonal=True))


def study(name, grid, bands, variants, rng=None):
    rng = rng or np.random.default_rng(0)
    A = D.dense_A(grid, bands)
    b = rng.standard_normal(A.shape[0])
    ilu = ilu0_dense(grid, A)
    rows = []
    for v in variants:
        B, x3s, x2s = dense_ntd(grid, bands, *v)
        try:
            ev = sla.eigh(A, B, eigvals_only=True)
            lo, hi = ev[0], ev[-1]
        except np.linalg.LinAlgError:
            w = np.linalg.eigvals(np.linalg.solve(B, A)).real
            lo, hi = float(w.min()), float(w.max())
        Binv = np.linalg.inv(B)
        it_ntd = cg_iters(A, lambda r: Binv @ r, b)

        def combo(r):
            y = ilu(r)
            return y + Binv @ (r - A @ y)
        it_c = cg_iters(A, combo, b, flexible=True)
        rows.append((name, v, lo, hi, indefiniteness(x3s), indefiniteness(x2s), it_ntd, it_c))
    return rows


VARIANTS = [("newton", "newton", "nested"), ("newton", "newton", "exact"),
            ("beta", "beta", "nested"), ("beta", "beta", "exact"),
            ("newton", "beta", "nested"), ("beta", "newton", "nested")]


def main(argv):
    from oracle import oracle as o
    from paper_1909_09771_gb300 import inputs as I
    sizes = [int(a) for a in argv] or [8, 12]
    print("variant = (level-3 X, level-2 X, inverse inside beta-hat); eigenvalues of B^-1 A; "
          "neg(X) = most negative eigenvalue of X / largest; iterations to 1e-8 (random b)")
    for n in sizes:
        cases = [(f"paper type {k}, {n}^3", I.workload_paper(k, n)) for k in (1, 2, 3)]
        cases.append((f"blocks 10^e e in [-3,3], {n}^3", I.random_small((n, n, n), 5, contrast_exp=3)))
        cases.append((f"GRF 10^(3g), {n}^3", I.workload_grf(seed=0, n=n)))
        for name, w in cases:
            bands = o.assemble(w["grid"], w["kappa"], w["bc"])
            for r in study(name, w["grid"], bands, VARIANTS):
                nm, v, lo, hi, n3, n2, itn, itc = r
                print(f"{nm:34s} {'/'.join(v):22s} lambda [{lo:9.3e}, {hi:9.3e}]  neg(X3) {n3:9.2e} "
                      f"neg(X2) {n2:9.2e}  CG B_NTD {itn:5d}  B_c {itc:4d}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
