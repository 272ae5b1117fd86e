"""Seeded synthetic inputs: cell-centred finite-volume discretisations of
-div(K grad u) = f on the unit square / cube (the model problem of Sec. 2,
Eq. (model) and Eq. (ls)).

This module produces the linear systems A x = b that both the CUDA path and
the CPU oracle consume.  It holds none of the multigrid method's arithmetic:
only random coefficient fields, the finite-volume assembly and CSR packing.

Discretisation (the same for every workload):
  * n_a cells along physical axis a, spacing h_a = 1 / n_a, cells numbered
    lexicographically with x fastest: idx = i + n_x (j + n_y k).
  * interior face between cells p, q along axis a:
        T = aniso_a * 2 K_p K_q / (K_p + K_q) / h_a^2   (harmonic mean)
    contributes +T to A_pp and A_qq and -T to A_pq = A_qp.
  * Dirichlet face with value g on cell p:  +2 aniso_a K_p / h_a^2 to A_pp and
    +2 aniso_a K_p g / h_a^2 to b_p.  No-flux faces contribute nothing.
  * CSR: int32 row_ptr / col, float64 val, columns sorted within each row.

Random fields follow the sum-of-cosines construction
    Z(x) = sigma sqrt(2/M) sum_m cos(k_m . x + phi_m),
    k_m ~ N(0, l^-2 I), phi_m ~ U[0, 2 pi),  K = exp(Z),
which has a Gaussian covariance with variance sigma^2 and correlation length l.
The modes come from numpy.random.default_rng(seed).  The field is evaluated
exactly through the separable form cos(k.x + phi) = Re(e^{i phi} prod_a
e^{i k_a x_a}), so a 512^3 field costs a few matrix products.
"""

from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Problem:
    """A CSR system A x = b plus the description needed to reproduce it."""

    name: str
    shape: tuple            # cells per physical axis, (n_x, n_y[, n_z])
    row_ptr: np.ndarray     # int32 [n+1]
    col: np.ndarray         # int32 [nnz]
    val: np.ndarray         # float64 [nnz]
    b: np.ndarray           # float64 [n]
    meta: dict

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def dim(self) -> int:
        return len(self.shape)


# ---------------------------------------------------------------------------
# random coefficient fields
# ---------------------------------------------------------------------------

def gaussian_field(shape: Sequence[int], variance: float, corr_len: float,
                   seed: int, modes: int = 1000) -> np.ndarray:
    """Sum-of-cosines Gaussian field at the cell centres.

    Returns an array in C order with the physical axes reversed (z, y, x), so
    that ``ravel()`` gives the lexicographic cell numbering.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    rng = np.random.default_rng(seed)
    k = rng.normal(0.0, 1.0 / corr_len, size=(modes, d))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    amp = np.sqrt(variance) * np.sqrt(2.0 / modes)
    centres = [(np.arange(m, dtype=np.float64) + 0.5) / m for m in shape]
    E = [np.exp(1j * np.outer(centres[a], k[:, a])) for a in range(d)]
    ex = E[0] * np.exp(1j * phi)[None, :]
    if d == 1:
        return amp * np.real(ex.sum(axis=1))
    if d == 2:
        return amp * np.real(E[1] @ ex.T)                     # (ny, nx)
    nx, ny, nz = shape
    out = np.empty((nz, ny, nx))
    # chunk along y so the (ny_chunk * nx, M) complex block stays ~0.5 GB
    yc = max(1, int(2 ** 25 // max(1, nx * modes)))
    for y0 in range(0, ny, yc):
        y1 = min(ny, y0 + yc)
        w = (E[1][y0:y1, None, :] * ex[None, :, :]).reshape(-1, modes)
        out[:, y0:y1, :] = amp * np.real(E[2] @ w.T).reshape(nz, y1 - y0, nx)
    return out


# ---------------------------------------------------------------------------
# finite-volume assembly
# ---------------------------------------------------------------------------

def cell_centres(phys_shape) -> list:
    """Coordinates of the cell centres of the unit square/cube, as arrays of
    the array shape (reversed physical axes), one per physical axis."""
    axes = [(np.arange(m) + 0.5) / m for m in phys_shape]
    grids = np.meshgrid(*axes[::-1], indexing="ij")     # array axes (z, y, x)
    return grids[::-1]                                  # physical order (x, y, z)


def _face_centres(phys_shape, pa, side, sl):
    """Coordinates of the boundary face centres of the cells in slice ``sl``
    (the low or high face normal to physical axis ``pa``)."""
    pts = [c[sl] for c in cell_centres(phys_shape)]
    pts[pa] = np.full_like(pts[pa], 0.0 if side == 0 else 1.0)
    return pts


def assemble_fv(K: np.ndarray, bc: Sequence, f: Optional[np.ndarray] = None,
                aniso: Optional[Sequence[float]] = None):
    """Assemble the cell-centred FV matrix for coefficient array ``K``.

    ``K`` has array axes (z, y, x) (reversed physical axes).  ``bc[a]`` is a
    pair (low, high) for physical axis a; each side is ``None`` (no flux), a
    float g (Dirichlet value) or a callable g(x, y, z) of the face-centre
    coordinates (Dirichlet data varying along the face).  ``aniso[a]`` multiplies every transmissibility
    of faces normal to physical axis a.  Returns (row_ptr, col, val, b).
    """
    K = np.asarray(K, dtype=np.float64)
    d = K.ndim
    phys_shape = K.shape[::-1]
    h = [1.0 / m for m in phys_shape]
    if aniso is None:
        aniso = [1.0] * d
    diag = np.zeros(K.shape)
    b = np.zeros(K.shape) if f is None else np.array(f, dtype=np.float64).reshape(K.shape)
    # T_minus[ax] holds, for each cell, the transmissibility of the face to its
    # lower neighbour along array axis ax (0 where there is none).
    t_minus = []
    for ax in range(d):
        pa = d - 1 - ax
        fac = aniso[pa] / (h[pa] * h[pa])
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        Kl, Kr = K[tuple(lo)], K[tuple(hi)]
        T = fac * (2.0 * Kl * Kr / (Kl + Kr))
        diag[tuple(lo)] += T
        diag[tuple(hi)] += T
        tm = np.zeros(K.shape)
        tm[tuple(hi)] = T
        t_minus.append(tm)
        for side, g in enumerate(bc[pa]):
            if g is None:
                continue
            sl = [slice(None)] * d
            sl[ax] = 0 if side == 0 else -1
            sl = tuple(sl)
            tb = 2.0 * fac * K[sl]
            diag[sl] += tb
            if callable(g):
                b[sl] += tb * g(*_face_centres(phys_shape, pa, side, sl))
            else:
                b[sl] += tb * float(g)
    n = K.size
    strides = [int(np.prod(K.shape[ax + 1:])) for ax in range(d)]
    nslot = 2 * d + 1
    cols = np.zeros((n, nslot), dtype=np.int64)
    vals = np.zeros((n, nslot))
    mask = np.zeros((n, nslot), dtype=bool)
    idx = np.arange(n, dtype=np.int64)
    # lower neighbours, slowest axis first (most negative column first)
    for s, ax in enumerate(range(d)):
        tm = t_minus[ax].ravel()
        has = np.zeros(K.shape, dtype=bool)
        hi = [slice(None)] * d
        hi[ax] = slice(1, None)
        has[tuple(hi)] = True
        has = has.ravel()
        cols[:, s] = idx - strides[ax]
        vals[:, s] = -tm
        mask[:, s] = has
    cols[:, d] = idx
    vals[:, d] = diag.ravel()
    mask[:, d] = True
    # upper neighbours, fastest axis first
    for s, ax in enumerate(reversed(range(d))):
        slot = d + 1 + s
        lo = [slice(None)] * d
        lo[ax] = slice(0, -1)
        has = np.zeros(K.shape, dtype=bool)
        has[tuple(lo)] = True
        has = has.ravel()
        tm_up = np.zeros(K.shape)
        # the face between cell p and its upper neighbour q is T_minus of q
        src = [slice(None)] * d
        src[ax] = slice(1, None)
        tm_up[tuple(lo)] = t_minus[ax][tuple(src)]
        cols[:, slot] = idx + strides[ax]
        vals[:, slot] = -tm_up.ravel()
        mask[:, slot] = has
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[mask].astype(np.int32)
    val = vals[mask]
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("nnz exceeds int32 range")
    return row_ptr.astype(np.int32), col, val, b.ravel()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def laplace2d_random_rhs(n: int = 64, seed: int = 0) -> Problem:
    """2D n x n, K = 1, u = 0 on every side, f ~ U[-1, 1] i.i.d. per cell."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, size=(n, n))
    K = np.ones((n, n))
    rp, ci, va, b = assemble_fv(K, bc=[(0.0, 0.0), (0.0, 0.0)], f=f)
    return Problem(f"laplace2d_{n}", (n, n), rp, ci, va, b,
                   dict(kind="laplace2d", n=n, seed=seed))


def lognormal3d(shape=(128, 128, 128), variance: float = 4.0,
                corr_len: float = 0.05, seed: int = 0) -> Problem:
    """3D, K = exp(Z), u = 1 at x = 0, u = 0 at x = 1, no flux elsewhere, f = 0."""
    shape = tuple(int(s) for s in shape)
    Z = gaussian_field(shape, variance, corr_len, seed)
    K = np.exp(Z)
    rp, ci, va, b = assemble_fv(K, bc=[(1.0, 0.0), (None, None), (None, None)])
    return Problem("lognormal3d_" + "x".join(map(str, shape)), shape, rp, ci, va, b,
                   dict(kind="lognormal3d", variance=variance, corr_len=corr_len,
                        seed=seed))


def layered3d(shape=(256, 256, 256), variance: float = 4.0, corr_len: float = 0.05,
              layers: int = 8, contrast: float = 1e-6, seed: int = 0) -> Problem:
    """Log-normal K overlaid with ``layers`` horizontal slabs of factor ``contrast``.

    Slab centres ~ U[0, 1], thickness ~ U[2h, 0.05] (h = 1 / n_z); boundary
    conditions as ``lognormal3d``.
    """
    shape = tuple(int(s) for s in shape)
    Z = gaussian_field(shape, variance, corr_len, seed)
    K = np.exp(Z)
    nz = shape[2]
    rng = np.random.default_rng(seed + 7919)
    zc = (np.arange(nz) + 0.5) / nz
    hz = 1.0 / nz
    for _ in range(layers):
        c = rng.uniform(0.0, 1.0)
        t = rng.uniform(2.0 * hz, max(2.0 * hz, 0.05))
        inside = np.abs(zc - c) <= 0.5 * t
        K[inside, :, :] *= contrast
    rp, ci, va, b = assemble_fv(K, bc=[(1.0, 0.0), (None, None), (None, None)])
    return Problem("layered3d_" + "x".join(map(str, shape)), shape, rp, ci, va, b,
                   dict(kind="layered3d", variance=variance, corr_len=corr_len,
                        layers=layers, contrast=contrast, seed=seed))


def anisotropic3d(shape=(512, 512, 512), variance: float = 6.0, corr_len: float = 0.02,
                  zfac: float = 1e-3, seed: int = 0) -> Problem:
    """K = exp(Z) diag(1, 1, zfac); boundary conditions as ``lognormal3d``."""
    shape = tuple(int(s) for s in shape)
    Z = gaussian_field(shape, variance, corr_len, seed)
    K = np.exp(Z)
    rp, ci, va, b = assemble_fv(K, bc=[(1.0, 0.0), (None, None), (None, None)],
                                aniso=[1.0, 1.0, zfac])
    return Problem("anisotropic3d_" + "x".join(map(str, shape)), shape, rp, ci, va, b,
                   dict(kind="anisotropic3d", variance=variance, corr_len=corr_len,
                        zfac=zfac, seed=seed))


def serving_request(seed: int, lo: int = 16, hi: int = 96) -> Problem:
    """One request of the serving stream: box sides ~ U{lo..hi} independently
    (16..96 for the serving workload), variance ~ U[1, 6], correlation length
    0.1, boundary conditions as ``lognormal3d``."""
    rng = np.random.default_rng(10_000 + seed)
    shape = tuple(int(s) for s in rng.integers(lo, hi + 1, size=3))
    variance = float(rng.uniform(1.0, 6.0))
    p = lognormal3d(shape, variance=variance, corr_len=0.1, seed=seed)
    p.meta.update(kind="serving", request=seed)
    return p


def poisson_exp3d(n: int) -> Problem:
    """Poisson problem of the paper's second machine (Sec. 5, helics3a):
    -Laplace u = f on the unit cube, u = g on the boundary, K = 1.  The printed
    right-hand side (6 - 4|x|) e^|x| matches no closed form with the printed
    boundary data e^|x|; this reads the pair as u = e^(|x|^2), for which
    -Laplace u = -(6 + 4 |x|^2) e^(|x|^2) exactly."""
    shape = (n, n, n)
    X, Y, Z = cell_centres(shape)
    r2 = X * X + Y * Y + Z * Z
    f = -(6.0 + 4.0 * r2) * np.exp(r2)
    g = lambda x, y, z: np.exp(x * x + y * y + z * z)
    rp, ci, va, b = assemble_fv(np.ones(shape[::-1]), bc=[(g, g)] * 3, f=f)
    return Problem("poisson_exp3d_%d" % n, shape, rp, ci, va, b,
                   dict(kind="poisson_exp3d", u_exact=np.exp(r2).ravel()))


def cube_in_cube3d(n: int) -> Problem:
    """Heterogeneous diffusion problem of the paper's Sec. 5 (after Griebel,
    Metsch and Schweitzer): K = 1e3 in the centred cube of width 0.8,
    K = 1e-2 in the eight corner cubes of width 0.1, K = 1 elsewhere.  The
    paper names Dirichlet conditions without values and no source; this
    takes u = 0 on the boundary and f = 1."""
    shape = (n, n, n)
    X, Y, Z = cell_centres(shape)
    K = np.ones(shape[::-1])
    inner = (np.abs(X - 0.5) < 0.4) & (np.abs(Y - 0.5) < 0.4) & (np.abs(Z - 0.5) < 0.4)
    K[inner] = 1e3
    corner = ((np.minimum(X, 1 - X) < 0.1) & (np.minimum(Y, 1 - Y) < 0.1)
              & (np.minimum(Z, 1 - Z) < 0.1))
    K[corner] = 1e-2
    rp, ci, va, b = assemble_fv(K, bc=[(0.0, 0.0)] * 3, f=np.ones(shape[::-1]))
    return Problem("cube_in_cube3d_%d" % n, shape, rp, ci, va, b, dict(kind="cube_in_cube3d"))


def hub_graph2d(n: int, degree: int = 24, seed: int = 0) -> Problem:
    """2D 5-point Laplacian (u = 0 on the boundary) plus one extra vertex
    coupled to ``degree`` random cells with weight 1 (symmetric, diagonally
    dominant): a sparse matrix with one long row, for kernels whose tiles are
    sized by the longest row."""
    rp, ci, va = grid_laplacian((n, n))
    N = n * n
    rng = np.random.default_rng(seed)
    nb = np.sort(rng.choice(N, size=degree, replace=False))
    rows, cols, vals = [], [], []
    for i in range(N):
        for k in range(rp[i], rp[i + 1]):
            rows.append(i); cols.append(int(ci[k]))
            vals.append(float(va[k]) + (1.0 if ci[k] == i and i in set(nb.tolist()) else 0.0))
    for j in nb:
        rows += [N, int(j)]; cols += [int(j), N]; vals += [-1.0, -1.0]
    rows.append(N); cols.append(N); vals.append(degree + 1.0)
    rp2, ci2, va2 = _coo_to_csr(N + 1, rows, cols, vals)
    b = rng.uniform(-1.0, 1.0, size=N + 1)
    return Problem("hub_graph2d_%d_%d" % (n, degree), (n, n), rp2, ci2, va2, b,
                   dict(kind="hub_graph2d", degree=degree, seed=seed))


def laplacian_1d(n: int) -> tuple:
    """tridiag(-1, 2, -1) of order n as CSR (a closed-form test matrix)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        rows.append(i); cols.append(i); vals.append(2.0)
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(-1.0)
    return _coo_to_csr(n, rows, cols, vals)


def grid_laplacian(shape: Sequence[int], weights: Optional[Sequence[float]] = None,
                   dirichlet_shift: float = 0.0) -> tuple:
    """Graph Laplacian of a structured grid (5-/7-point), optionally with
    per-axis weights and ``dirichlet_shift`` added to every diagonal entry so the
    matrix is SPD.  Lexicographic numbering, x fastest."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    if weights is None:
        weights = [1.0] * d
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[:a])) for a in range(d)]
    rows, cols, vals = [], [], []
    for idx in range(n):
        coord = [(idx // strides[a]) % shape[a] for a in range(d)]
        diag = dirichlet_shift
        entries = []
        for a in range(d):
            if coord[a] > 0:
                entries.append((idx - strides[a], -weights[a]))
                diag += weights[a]
            if coord[a] < shape[a] - 1:
                entries.append((idx + strides[a], -weights[a]))
                diag += weights[a]
        entries.append((idx, diag))
        for j, v in sorted(entries):
            rows.append(idx); cols.append(j); vals.append(v)
    return _coo_to_csr(n, rows, cols, vals)


def _coo_to_csr(n, rows, cols, vals):
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int32)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return rp, cols, vals


def config_problem(name: str, scale: Optional[Sequence[int]] = None, seed: int = 0) -> Problem:
    """The named workloads, optionally at a reduced grid ``scale``.

    ``laplace2d``      2D 64^2, K = 1, u = 0 on the boundary, f ~ U[-1, 1]
    ``lognormal``      3D 128^3, variance 4, correlation length 0.05
    ``layered``        3D 256^3, variance 4, 8 slabs of contrast 1e-6
    ``anisotropic``    3D 512^3, variance 6, correlation length 0.02, z x 1e-3
    """
    if name == "laplace2d":
        n = 64 if scale is None else int(scale[0])
        return laplace2d_random_rhs(n, seed)
    if name == "lognormal":
        return lognormal3d((128,) * 3 if scale is None else scale, seed=seed)
    if name == "layered":
        return layered3d((256,) * 3 if scale is None else scale, seed=seed)
    if name == "anisotropic":
        return anisotropic3d((512,) * 3 if scale is None else scale, seed=seed)
    raise KeyError(name)
