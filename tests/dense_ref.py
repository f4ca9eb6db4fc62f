"""Dense-matrix helpers for the pins (small grids only).

They build matrices from band arrays with numpy and the twisted block
structure of Sec. II-A; they share no code with the oracle's sweeps.
"""
import numpy as np


def dense_A(grid, bands):
    nx, ny, nz = grid
    n = nx * ny * nz
    d, cx, cy, cz = bands
    A = np.diag(np.asarray(d, dtype=np.float64))
    for c, s in ((cx, 1), (cy, nx), (cz, nx * ny)):
        idx = np.arange(n - s)
        A[idx, idx + s] = c[: n - s]
        A[idx + s, idx] = c[: n - s]
    return A


def twisted_lower(nb, bs, coupling):
    """Twisted block-lower matrix L for nb blocks of size bs: block rows
    q = 1..m take the coupling to block q-1, block rows q = m..nb-2 take the
    coupling to block q+1 (m = floor((nb-1)/2)).  coupling[q*bs + e] couples
    entry e of block q with entry e of block q+1."""
    n = nb * bs
    L = np.zeros((n, n))
    m = (nb - 1) // 2
    for q in range(1, m + 1):
        for e in range(bs):
            L[q * bs + e, (q - 1) * bs + e] = coupling[(q - 1) * bs + e]
    for q in range(m, nb - 1):
        for e in range(bs):
            L[q * bs + e, (q + 1) * bs + e] = coupling[q * bs + e]
    return L


def tridiag(diag, off):
    T = np.diag(diag)
    if len(diag) > 1:
        T += np.diag(off[:-1], 1) + np.diag(off[:-1], -1)
    return T


def line_T_from_pivots(M, off):
    """T = (M + L1) M^{-1} (M + U1) for one line (Sec. II-A, level 1)."""
    n = len(M)
    L1 = twisted_lower(n, 1, off)
    Md = np.diag(M)
    return (Md + L1) @ np.diag(1.0 / M) @ (Md + L1.T)


def plane_BP(nx, ny, Td, To, Py, M=None):
    """B_P = (T + L2) T^{-1} (T + U2) for one plane; T = blockdiag of the line
    tridiagonals (Td, To), or of (M + L1)M^{-1}(M + U1) when pivots M are given."""
    n = nx * ny
    T = np.zeros((n, n))
    for k in range(ny):
        s = slice(k * nx, (k + 1) * nx)
        if M is None:
            T[s, s] = tridiag(Td[s], To[s])
        else:
            T[s, s] = line_T_from_pivots(M[s], To[s])
    L2 = twisted_lower(ny, nx, Py)
    return (T + L2) @ np.linalg.inv(T) @ (T + L2.T)


def dense_B(grid, f, use_pivots=True):
    """B = (B_P + L3) B_P^{-1} (B_P + U3) from the stored setup output."""
    nx, ny, nz = grid
    nxy = nx * ny
    n = nxy * nz
    BP = np.zeros((n, n))
    for i in range(nz):
        s = slice(i * nxy, (i + 1) * nxy)
        BP[s, s] = plane_BP(nx, ny, f.Td[s], f.To[s], f.Py[s], f.M[s] if use_pivots else None)
    L3 = twisted_lower(nz, nxy, f.l3)
    return (BP + L3) @ np.linalg.inv(BP) @ (BP + L3.T), BP


def plane_P(nx, ny, Pd, Px, Py):
    n = nx * ny
    P = np.diag(Pd.copy())
    for c, s in ((Px, 1), (Py, nx)):
        idx = np.arange(n - s)
        P[idx, idx + s] = c[: n - s]
        P[idx + s, idx] = c[: n - s]
    return P
