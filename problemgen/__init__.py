"""Seeded synthetic inputs for the regularized least-squares solver.

This module produces the *inputs* of the method only: phantoms x_true,
forward operators A (a ray-length CSR matrix for parallel-beam CT, or a
Gaussian point-spread function applied as a zero-boundary correlation),
noisy data b = A x_true + noise, weight vectors D, and lambda grids.  It
contains none of the solver's arithmetic and is imported both by the CPU
oracle (``oracle/``) and by the GPU path's tests and benchmark, which is the
only code the two sides share.

Conventions (Sec. 2 of the paper):
  * An image is n_v x n_h.  Vectors are stored column-major: pixel (i, j)
    (row i from the top, column j from the left) has index i + j * n_v, the
    vectorisation implied by the Kronecker form of the gradient.
  * Random numbers come from numpy's PCG64 bit generator (O'Neill 2014)
    seeded with the workload's integer seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng", "phantom_rectangles", "phantom_ellipses", "phantom_mixed",
    "gaussian_psf", "blur_csr", "blur_apply", "ct_csr", "add_noise",
    "CSR", "Problem", "make_problem", "WORKLOADS", "logspace_increasing",
    "random_weights",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# Phantoms (painter's order: later shapes overwrite earlier ones, background 0)
# --------------------------------------------------------------------------
def _grid(n_v: int, n_h: int):
    i = np.arange(n_v, dtype=np.float64)[:, None] + 0.5
    j = np.arange(n_h, dtype=np.float64)[None, :] + 0.5
    return i, j


def phantom_rectangles(n_v, n_h, count, seed, lo=0.0, hi=1.0):
    """Axis-aligned constant-intensity rectangles; returns an (n_v, n_h) image."""
    g = rng(seed)
    img = np.zeros((n_v, n_h))
    i, j = _grid(n_v, n_h)
    for _ in range(count):
        ci, cj = g.uniform(0, n_v), g.uniform(0, n_h)
        hi_, hj = g.uniform(n_v / 16, n_v / 4), g.uniform(n_h / 16, n_h / 4)
        val = g.uniform(lo, hi)
        m = (np.abs(i - ci) <= hi_) & (np.abs(j - cj) <= hj)
        img[m] = val
    return img


def phantom_ellipses(n_v, n_h, count, seed, lo=0.1, hi=1.0):
    """Rotated constant-intensity ellipses; returns an (n_v, n_h) image."""
    g = rng(seed)
    img = np.zeros((n_v, n_h))
    i, j = _grid(n_v, n_h)
    for _ in range(count):
        ci, cj = g.uniform(0, n_v), g.uniform(0, n_h)
        a, b = g.uniform(n_v / 16, n_v / 4), g.uniform(n_h / 16, n_h / 4)
        th = g.uniform(0, math.pi)
        val = g.uniform(lo, hi)
        di, dj = i - ci, j - cj
        u = di * math.cos(th) + dj * math.sin(th)
        v = -di * math.sin(th) + dj * math.cos(th)
        img[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = val
    return img


def phantom_mixed(n_v, n_h, count, seed, lo=0.0, hi=1.0):
    """Rectangles and ellipses alternately (piecewise-constant image)."""
    g = rng(seed)
    img = np.zeros((n_v, n_h))
    i, j = _grid(n_v, n_h)
    for k in range(count):
        ci, cj = g.uniform(0, n_v), g.uniform(0, n_h)
        a, b = g.uniform(n_v / 16, n_v / 4), g.uniform(n_h / 16, n_h / 4)
        th = g.uniform(0, math.pi)
        val = g.uniform(lo, hi)
        di, dj = i - ci, j - cj
        if k % 2 == 0:
            m = (np.abs(di) <= a) & (np.abs(dj) <= b)
        else:
            u = di * math.cos(th) + dj * math.sin(th)
            v = -di * math.sin(th) + dj * math.cos(th)
            m = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        img[m] = val
    return img


def vec(img: np.ndarray) -> np.ndarray:
    """Column-major vectorisation of an (n_v, n_h) image."""
    return np.asarray(img, dtype=np.float64).reshape(-1, order="F").copy()


def unvec(x: np.ndarray, n_v: int, n_h: int) -> np.ndarray:
    return np.asarray(x).reshape((n_v, n_h), order="F")


# --------------------------------------------------------------------------
# Blur: Gaussian PSF, zero boundary (rows truncated, not renormalised)
# --------------------------------------------------------------------------
def gaussian_psf(radius: int, sigma: float) -> np.ndarray:
    """(2r+1)^2 Gaussian exp(-(u^2+v^2)/(2 sigma^2)), normalised to sum 1."""
    u = np.arange(-radius, radius + 1, dtype=np.float64)
    g1 = np.exp(-(u ** 2) / (2.0 * sigma * sigma))
    psf = np.outer(g1, g1)
    return psf / psf.sum()


def separable_psf(n_v: int, n_h: int, band_v: int = 7, band_h: int = 8, s_v: float = 1.25,
                  s_h: float = 1.5) -> np.ndarray:
    """Anisotropic separable blur of the deblurring experiment (Sec. 4): the
    product of a vertical and a horizontal 1-D Gaussian, each truncated to
    |offset| < band and with width s * side / 64 pixels, each normalised so
    that its two-sided sum is 1.  Returns the (2 band_v - 1) x (2 band_h - 1)
    PSF (vertical offsets along rows)."""
    def one_d(band, sigma):
        half = np.exp(-(np.arange(band, dtype=np.float64) ** 2) / (2.0 * sigma * sigma))
        half /= 2.0 * half.sum() - half[0]
        return np.concatenate([half[:0:-1], half])
    return np.outer(one_d(band_v, s_v * n_v / 64.0), one_d(band_h, s_h * n_h / 64.0))


def blur_apply(img: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """(A x)(i, j) = sum_{u,v} psf[u+r_v, v+r_h] x(i+u, j+v), zero outside."""
    from scipy.ndimage import correlate
    return correlate(np.asarray(img, dtype=np.float64), psf, mode="constant", cval=0.0)


@dataclass
class CSR:
    m: int
    n: int
    row_ptr: np.ndarray  # int64, m+1
    col: np.ndarray      # int32, nnz
    val: np.ndarray      # float32 or float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self, dtype=np.float64):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.astype(dtype), self.col.astype(np.int64),
                              self.row_ptr.astype(np.int64)), shape=(self.m, self.n))


def blur_csr(n_v: int, n_h: int, psf: np.ndarray, dtype=np.float64) -> CSR:
    """The zero-boundary correlation with ``psf`` as an explicit CSR matrix."""
    kh, kw = psf.shape
    rv, rh = kh // 2, kw // 2
    rows, cols, vals = [], [], []
    ii = np.arange(n_v)
    jj = np.arange(n_h)
    I, J = np.meshgrid(ii, jj, indexing="ij")
    out_idx = (I + J * n_v).reshape(-1, order="F")
    for du in range(-rv, rv + 1):
        for dv in range(-rh, rh + 1):
            w = psf[du + rv, dv + rh]
            Ii, Jj = I + du, J + dv
            ok = (Ii >= 0) & (Ii < n_v) & (Jj >= 0) & (Jj < n_h)
            okf = ok.reshape(-1, order="F")
            src = (Ii + Jj * n_v).reshape(-1, order="F")
            rows.append(out_idx[okf]); cols.append(src[okf])
            vals.append(np.full(okf.sum(), w))
    import scipy.sparse as sp
    n = n_v * n_h
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    M.sort_indices()
    return CSR(n, n, M.indptr.astype(np.int64), M.indices.astype(np.int32),
               M.data.astype(dtype))


# --------------------------------------------------------------------------
# Parallel-beam CT: exact ray/pixel intersection lengths (Siddon 1985)
# --------------------------------------------------------------------------
def ct_csr(N: int, n_angles: int, n_bins: int, dtype=np.float32,
           angles_deg=None) -> CSR:
    """Ray-length matrix for an N x N image on the square [-N/2, N/2]^2.

    Angles theta_a = a * 180 / n_angles degrees (or ``angles_deg``), detector
    offsets s_b = b - (n_bins - 1) / 2 pixels.  Ray (a, b) is the line
    {p : p . (cos t, sin t) = s_b}; rows are angle-major (row = a*n_bins + b).
    Pixel (i, j) covers x in [-N/2 + j, -N/2 + j + 1] and
    y in [N/2 - i - 1, N/2 - i].  Zero-length intersections are dropped.
    """
    if angles_deg is None:
        angles_deg = np.arange(n_angles, dtype=np.float64) * 180.0 / n_angles
    angles = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    half = N / 2.0
    lines = np.arange(N + 1, dtype=np.float64) - half
    s = np.arange(n_bins, dtype=np.float64) - (n_bins - 1) / 2.0
    row_counts = []
    cols_all, vals_all = [], []
    eps = 1e-9
    for th in angles:
        c, sn = math.cos(th), math.sin(th)
        px, py = s * c, s * sn            # foot point of each ray
        dx, dy = -sn, c                   # unit direction
        ts = []
        big = 1e30
        if abs(dx) > 1e-12:
            tx = (lines[None, :] - px[:, None]) / dx
            ts.append(tx)
            txa, txb = tx[:, 0], tx[:, -1]
            tx_lo, tx_hi = np.minimum(txa, txb), np.maximum(txa, txb)
        else:
            inside = (px >= -half) & (px <= half)
            tx_lo = np.where(inside, -big, big)
            tx_hi = np.where(inside, big, -big)
        if abs(dy) > 1e-12:
            ty = (lines[None, :] - py[:, None]) / dy
            ts.append(ty)
            tya, tyb = ty[:, 0], ty[:, -1]
            ty_lo, ty_hi = np.minimum(tya, tyb), np.maximum(tya, tyb)
        else:
            inside = (py >= -half) & (py <= half)
            ty_lo = np.where(inside, -big, big)
            ty_hi = np.where(inside, big, -big)
        t0 = np.maximum(tx_lo, ty_lo)
        t1 = np.minimum(tx_hi, ty_hi)
        T = np.concatenate(ts + [t0[:, None], t1[:, None]], axis=1)
        T = np.clip(T, t0[:, None], np.maximum(t0, t1)[:, None])
        T.sort(axis=1)
        L = np.diff(T, axis=1)
        mid = 0.5 * (T[:, 1:] + T[:, :-1])
        live = L > eps
        mid = np.where(live, mid, 0.0)
        mx = px[:, None] + mid * dx
        my = py[:, None] + mid * dy
        jcol = np.floor(np.clip(mx + half, -1.0, N + 1.0)).astype(np.int64)
        irow = np.floor(np.clip(half - my, -1.0, N + 1.0)).astype(np.int64)
        ok = live & (jcol >= 0) & (jcol < N) & (irow >= 0) & (irow < N)
        idx = irow + jcol * N
        for r in range(n_bins):
            okr = ok[r]
            row_counts.append(int(okr.sum()))
            cols_all.append(idx[r][okr])
            vals_all.append(L[r][okr])
    m = len(row_counts)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(row_counts)
    col = np.concatenate(cols_all).astype(np.int32)
    val = np.concatenate(vals_all).astype(dtype)
    return CSR(m, N * N, row_ptr, col, val)


# --------------------------------------------------------------------------
# Noise, lambda grids, weights
# --------------------------------------------------------------------------
def add_noise(b_true: np.ndarray, level: float, seed: int) -> np.ndarray:
    """b = b_true + level * ||b_true|| * e / ||e||, e ~ N(0, I)."""
    e = rng(seed).standard_normal(b_true.shape[0])
    return b_true + level * np.linalg.norm(b_true) * e / np.linalg.norm(e)


def logspace_increasing(lo_exp: float, hi_exp: float, count: int) -> np.ndarray:
    return np.logspace(lo_exp, hi_exp, count)


def random_weights(n_edges: int, seed: int, d_min=1e-3) -> np.ndarray:
    return rng(seed).uniform(d_min, 1.0, n_edges)


def n_edges(n_v: int, n_h: int) -> int:
    return n_h * (n_v - 1) + (n_h - 1) * n_v


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    n_v: int
    n_h: int
    kind: str                     # "csr" or "stencil"
    A: CSR | None
    psf: np.ndarray | None
    x_true: np.ndarray            # (n, n_rhs)
    b: np.ndarray                 # (m, n_rhs)
    lambdas: np.ndarray           # increasing
    levels: int
    tol: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.n_v * self.n_h

    @property
    def m(self):
        return self.A.m if self.A is not None else self.n


def _forward(problem_kind, A, psf, img):
    if problem_kind == "csr":
        return A.to_scipy() @ vec(img)
    return vec(blur_apply(img, psf))


def make_problem(name: str, size: int | None = None, n_rhs: int | None = None) -> Problem:
    """Build one of the named synthetic workloads (``WORKLOADS``).

    ``size`` overrides the image side (used by tests to run a workload's
    recipe at a reduced size); ``n_rhs`` overrides the number of phantoms.
    """
    w = WORKLOADS[name]
    N = size or w["side"]
    nr = n_rhs or w.get("n_rhs", 1)
    kind = w["kind"]
    A = psf = None
    if w["op"] == "blur_csr":
        psf = gaussian_psf(w["radius"], w["sigma"])
        A = blur_csr(N, N, psf, dtype=np.float64)
        kind = "csr"
    elif w["op"] == "blur":
        psf = gaussian_psf(w["radius"], w["sigma"])
    elif w["op"] == "blur_aniso":
        psf = separable_psf(N, N)
    elif w["op"] == "ct":
        nb = w["bins"] if size is None else int(2 * math.ceil(N * 1.42 / 2) - 1)
        if "angles_deg" in w:  # fixed angle set, whatever the size
            A = ct_csr(N, len(w["angles_deg"]), nb, dtype=np.float32, angles_deg=w["angles_deg"])
        else:
            na = w["angles"] if size is None else max(8, round(w["angles"] * N / w["side"]))
            A = ct_csr(N, na, nb, dtype=np.float32)
    xs, bs = [], []
    for r in range(nr):
        seed = w["seed"] + r
        if w["phantom"] == "rect":
            img = phantom_rectangles(N, N, w["count"], seed, 0.0, 1.0)
        elif w["phantom"] == "ellipse":
            img = phantom_ellipses(N, N, w["count"], seed, 0.1, 1.0)
        else:
            img = phantom_mixed(N, N, w["count"], seed, 0.0, 1.0)
        bt = _forward(kind, A, psf, img)
        xs.append(vec(img))
        bs.append(add_noise(bt, w["noise"], w["noise_seed"] + r))
    lam = logspace_increasing(w["lam_lo"], w["lam_hi"], w["n_lambda"])
    if "lambdas" in w:
        lam = np.asarray(w["lambdas"], dtype=np.float64)
    levels = w["levels"]
    if size is not None and levels:
        levels = max(1, levels - int(round(math.log2(w["side"] / N))))
    return Problem(name, N, N, kind, A, psf, np.stack(xs, 1), np.stack(bs, 1), lam,
                   levels, w["tol"], dict(w))


#   side: image side; kind: csr | stencil; levels: 0 = coarsen until <= 16
WORKLOADS = {
    # 32x32 deblurring, 4 rectangles, 9x9 Gaussian sigma 1.5 as an FP64 CSR
    # matrix, 1% noise, D = I, one lambda = 0.05, 3-level V-cycle, tol 1e-10.
    "deblur32_csr": dict(side=32, kind="csr", op="blur_csr", radius=4, sigma=1.5,
                         phantom="rect", count=4, seed=0, noise=0.01, noise_seed=1000,
                         lam_lo=math.log10(0.05), lam_hi=math.log10(0.05), n_lambda=1,
                         lambdas=[0.05], levels=3, tol=1e-10),
    # 256x256 CT, 10 ellipses, 180 angles x 363 bins ray-length CSR (FP32
    # values, int32 columns), 1% noise, 20 lambdas in [1e-4, 1], outer loop.
    "ct256": dict(side=256, kind="csr", op="ct", angles=180, bins=363,
                  phantom="ellipse", count=10, seed=1, noise=0.01, noise_seed=1001,
                  lam_lo=-4.0, lam_hi=0.0, n_lambda=20, levels=0, tol=1e-6,
                  max_outer=15),
    # 512x512 deblurring, 19x19 Gaussian sigma 3 matrix-free, 4 phantoms,
    # 32 lambdas in [1e-5, 1], 5 outer iterations, 6 levels.
    "deblur512": dict(side=512, kind="stencil", op="blur", radius=9, sigma=3.0,
                      phantom="mixed", count=8, seed=2, n_rhs=4, noise=0.01,
                      noise_seed=1002, lam_lo=-5.0, lam_hi=0.0, n_lambda=32, levels=6,
                      tol=1e-6, max_outer=5),
    # Workload variants of Sec. 4: limited-angle CT (angles 0, 2, ..., 130
    # degrees) and deblurring with the anisotropic separable blur, both on
    # piecewise-constant phantoms standing in for the paper's grains image.
    "ct256_limited": dict(side=256, kind="csr", op="ct", angles=66, bins=363,
                          angles_deg=[2.0 * a for a in range(66)], phantom="mixed", count=20,
                          seed=11, noise=0.01, noise_seed=1011, lam_lo=-4.0, lam_hi=0.0,
                          n_lambda=20, levels=0, tol=1e-6, max_outer=15),
    "deblur256_aniso": dict(side=256, kind="stencil", op="blur_aniso", phantom="mixed", count=20,
                            seed=12, noise=0.01, noise_seed=1012, lam_lo=-5.0, lam_hi=0.0,
                            n_lambda=32, levels=0, tol=1e-6, max_outer=15),
    # 2048x2048 deblurring, 31x31 Gaussian sigma 5, 64 lambdas in [1e-6, 1],
    # 10 levels, 2% noise.
    "deblur2048": dict(side=2048, kind="stencil", op="blur", radius=15, sigma=5.0,
                       phantom="mixed", count=20, seed=9, noise=0.02, noise_seed=1009,
                       lam_lo=-6.0, lam_hi=0.0, n_lambda=64, levels=10, tol=1e-6),
}
