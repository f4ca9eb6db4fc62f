"""Seeded synthetic inputs (diffusion coefficient fields, right-hand sides,
boundary flags) for the five workloads.  This module holds none of the
method's arithmetic: it only draws numbers.  It is the one module that both
the CUDA path's tests/benchmark and the CPU oracle's tests take inputs from.

Index order is x fastest: a = x + nx*(y + ny*z).  Draw order: kappa
parameters first, then right-hand sides.  Every generator takes an explicit
seed and uses numpy's default_rng(seed).

Workloads (unit cube, Dirichlet u=0 on the z=0 and z=1 faces, Neumann on the
x and y faces, unless stated):
  blocks32     32^3, kappa = 10^e on a 4x4x4 block partition, e uniform integer
               in [-3, 3]; b ~ N(0,1)
  layered128   128^3, 16 z-layers alternating kappa 1 and 1e6, eight 16^3
               inclusions of kappa 1e-3; b = h^3 (f = 1 scaled by cell volume)
  grf350       350^3, kappa = 10^(3 g), g a Gaussian random field with
               correlation length 0.1, normalised, clipped to [-1, 1]; b ~ N(0,1)
  batched      64 instances, each nx,ny,nz uniform in [48, 160], kappa = 10^e on
               an 8x8x8 block partition, 4 right-hand sides N(0,1) each
  grf_train    64^3 GRF instances with contrast 10^4 (kappa = 10^(2 g))
  paper<T>_<n> the paper's own test problems (Sec. IV, "Test Matrices"): n^3,
               Dirichlet u=0 on all six faces, kappa of type T = 1 (skyscrapers
               with checkerboard jumps), 2 (a ring of kappa 1e3), 3 (Poisson);
               b = h^3 (f = 1 scaled by cell volume; the paper does not state f)
"""
from __future__ import annotations

import numpy as np

# x-, x+, y-, y+, z-, z+ ; 0 = Dirichlet, 1 = Neumann
BC_Z_DIRICHLET = (1, 1, 1, 1, 0, 0)
BC_ALL_DIRICHLET = (0, 0, 0, 0, 0, 0)


def kappa_blocks(grid, nblocks, seed, emin=-3, emax=3, rng=None):
    """kappa = 10^e, e an integer uniform in [emin, emax] per block of an
    nblocks^3 partition; a cell with coordinate c along an axis of n cells is
    in block floor(nblocks * c / n)."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed) if rng is None else rng
    e = rng.integers(emin, emax + 1, size=(nblocks, nblocks, nblocks))  # [bz, by, bx]
    bx = (nblocks * np.arange(nx)) // nx
    by = (nblocks * np.arange(ny)) // ny
    bz = (nblocks * np.arange(nz)) // nz
    ee = e[bz[:, None, None], by[None, :, None], bx[None, None, :]]
    return np.power(10.0, ee).reshape(-1)


def kappa_layered(n, seed, layers=16, hi=1e6, lo=1.0, incl=8, incl_size=16, incl_val=1e-3, rng=None):
    """z-layers of n/layers cells alternating lo (even layer, from z=0) and hi,
    then `incl` cubes of incl_size^3 cells with kappa = incl_val at corners drawn
    uniformly in [0, n - incl_size] (later ones overwrite earlier ones)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    k = np.empty((n, n, n))
    th = n // layers
    for z in range(n):
        k[z] = lo if (z // th) % 2 == 0 else hi
    corners = rng.integers(0, n - incl_size + 1, size=(incl, 3))
    for cz, cy, cx in corners:
        k[cz:cz + incl_size, cy:cy + incl_size, cx:cx + incl_size] = incl_val
    return k.reshape(-1)


def gaussian_field(n, seed, ell=0.1, rng=None, chunk=None):
    """Seeded Gaussian random field on an n^3 periodic grid of the unit cube:
    white noise N(0,1) per cell filtered by a Gaussian kernel of standard
    deviation ell/sqrt(2) (covariance ~ exp(-r^2 / (2 ell^2)) up to the periodic
    wrap), normalised to unit sample standard deviation.  Returned with x
    fastest as float64, shape (n^3,)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    w = rng.standard_normal((n, n, n), dtype=np.float64)
    sigma = ell / np.sqrt(2.0)
    f = np.fft.fftfreq(n)  # cycles per cell
    # Gaussian transfer function exp(-2 pi^2 sigma^2 k^2) with k in cycles per unit length
    g1 = np.exp(-2.0 * np.pi ** 2 * (sigma * n) ** 2 * f ** 2)
    W = np.fft.rfftn(w)
    del w
    g_last = g1[: W.shape[2]]
    W *= g1[:, None, None]
    W *= g1[None, :, None]
    W *= g_last[None, None, :]
    g = np.fft.irfftn(W, s=(n, n, n), axes=(0, 1, 2))
    del W
    g -= g.mean()
    g /= g.std()
    return g.reshape(-1)


def kappa_grf(n, seed, exponent=3.0, ell=0.1, rng=None):
    """kappa = 10^(exponent * clip(g, -1, 1)), g = gaussian_field."""
    g = gaussian_field(n, seed, ell=ell, rng=rng)
    np.clip(g, -1.0, 1.0, out=g)
    return np.power(10.0, exponent * g)


def rhs_normal(npts, rng):
    return rng.standard_normal(npts)


def workload_blocks32(seed=0, n=32):
    rng = np.random.default_rng(seed)
    grid = (n, n, n)
    kappa = kappa_blocks(grid, 4, seed, rng=rng)
    b = rhs_normal(n ** 3, rng)
    return dict(name=f"blocks{n}", grid=grid, kappa=kappa, bc=BC_Z_DIRICHLET, b=b)


def workload_layered128(seed=0, n=128):
    rng = np.random.default_rng(seed)
    grid = (n, n, n)
    kappa = kappa_layered(n, seed, rng=rng, layers=16, incl_size=max(1, n // 8))
    h = 1.0 / n
    b = np.full(n ** 3, h ** 3)
    return dict(name=f"layered{n}", grid=grid, kappa=kappa, bc=BC_Z_DIRICHLET, b=b)


def kappa_paper(kind, n):
    """Coefficient of the paper's test matrix type `kind` (Sec. IV, "Test
    Matrices") at the cell centres x = ((i+1/2)/n, (j+1/2)/n, (k+1/2)/n) of
    an n^3 unit cube, x fastest:
      1: 10^3 ([10 x_2] + 1) where [10 x_i] is even for i = 1, 2, 3, else 1
         ([.] the integer part, x_2 the y coordinate);
      2: 10^3 on the shell 1/(2 sqrt 2) <= |x - c| <= 1/2, c the cube centre,
         else 1;
      3: 1."""
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")  # arrays [z, y, x]: x fastest when raveled
    if kind == 1:
        fx, fy, fz = np.floor(10 * x), np.floor(10 * y), np.floor(10 * z)
        even = (fx % 2 == 0) & (fy % 2 == 0) & (fz % 2 == 0)
        k = np.where(even, 1e3 * (fy + 1.0), 1.0)
    elif kind == 2:
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        k = np.where((r >= 1.0 / (2.0 * np.sqrt(2.0))) & (r <= 0.5), 1e3, 1.0)
    elif kind == 3:
        k = np.ones((n, n, n))
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(k, dtype=np.float64).ravel()


def workload_paper(kind, n):
    """The paper's test problem of type `kind` on n^3 (Sec. IV): all faces
    Dirichlet, b = h^3 (f = 1)."""
    h = 1.0 / n
    return dict(name=f"paper{kind}_{n}", grid=(n, n, n), kappa=kappa_paper(kind, n),
                bc=BC_ALL_DIRICHLET, b=np.full(n ** 3, h ** 3))


def workload_grf(seed=0, n=350, exponent=3.0):
    rng = np.random.default_rng(seed)
    grid = (n, n, n)
    kappa = kappa_grf(n, seed, exponent=exponent, rng=rng)
    b = rhs_normal(n ** 3, rng)
    return dict(name=f"grf{n}", grid=grid, kappa=kappa, bc=BC_Z_DIRICHLET, b=b)


def batched_grids(seed=0, count=64, lo=48, hi=160):
    """The grids of the batched workload's instances (the first draw of each
    instance's generator), without generating their fields."""
    return [tuple(int(v) for v in np.random.default_rng(seed + i).integers(lo, hi + 1, size=3))
            for i in range(count)]


def workload_batched(seed=0, count=64, nrhs=4, lo=48, hi=160, indices=None):
    """Instance i uses seed + i: sizes first, then its 8x8x8-block kappa, then
    its nrhs right-hand sides.  indices: generate only these instances (in the
    order given); default all `count`."""
    out = []
    for i in (range(count) if indices is None else indices):
        rng = np.random.default_rng(seed + i)
        nx, ny, nz = (int(v) for v in rng.integers(lo, hi + 1, size=3))
        kappa = kappa_blocks((nx, ny, nz), 8, None, rng=rng)
        bs = np.stack([rhs_normal(nx * ny * nz, rng) for _ in range(nrhs)])
        out.append(dict(name=f"inst{i}", grid=(nx, ny, nz), kappa=kappa, bc=BC_Z_DIRICHLET, b=bs))
    return out


def random_small(grid, seed, contrast_exp=3, bc=BC_Z_DIRICHLET, per_cell=False):
    """Small seeded instance for tests: block (2x2x2) or per-cell kappa
    10^U[-c, c], b ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(grid))
    if per_cell:
        kappa = np.power(10.0, rng.uniform(-contrast_exp, contrast_exp, n))
    else:
        kappa = kappa_blocks(grid, 2, None, emin=-contrast_exp, emax=contrast_exp, rng=rng)
    b = rng.standard_normal(n)
    return dict(name=f"rand{grid}", grid=tuple(grid), kappa=kappa, bc=tuple(bc), b=b)


def lanczos_start(n, seed):
    """Start vector of a Lanczos run: N(0,1) per cell from default_rng(seed)."""
    return np.random.default_rng(seed).standard_normal(int(n))


def workload_learned_train(count=2000, n=64, seed0=10_000, exponent=2.0):
    """Training instances of the learned filter: instance i is the n^3 GRF of
    seed seed0 + i with kappa = 10^(exponent g) (contrast 10^(2 exponent))."""
    for i in range(count):
        yield workload_grf(seed=seed0 + i, n=n, exponent=exponent)
