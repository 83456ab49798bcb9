"""Seeded synthetic inputs shared by the tests, the bench and the CPU baseline.

This module holds none of the method's arithmetic: operator parameters and random
right-hand sides only.  Each side (the CUDA path and the oracle) builds its own operator
from these parameters.  Random numbers: numpy Generator(PCG64(seed)), N(0, 1), laid out
column by column (column c of B is one contiguous draw of n numbers), seed
20140707 + workload index.

Workloads (the paper's experiments use nu = 14 CF poles, Section 5; the block sizes, grid
sizes and times below are synthetic stand-ins for the paper's own matrices):
  tridiag-1d   A = t (n+1)^2 tridiag(1, -2, 1), n = 2000, t = 1, p = 4, m = 10, tol 1e-10
  cd2d-256     t (0.1 Laplacian_h - (1, 1) . grad_h) on a 256 x 256 interior grid,
               n = 65536, p = 8, t in {1e-3, 1e-2, 1e-1}, m = 10
  toeplitz-1m  t T, T symmetric Toeplitz with first column a_0 = -2 - c, a_k = 1/(1+k)^2
               (1 <= k <= 256), c = 0, n = 2^20, p = 16, t = 1, m = 10
  toeplitz-frac t T, T the symmetric part of Example 5.4's fractional diffusion matrix
               (beta = 1.8, fractional_column), n = 2^17, p = 2, t = 0.01, m = 30, k = 30, tol 1e-10
  batched3d-64 64 independent instances t (Laplacian_h - v . grad_h) on N_x x N_y x N_z grids,
               N_d uniform in {32..96} per axis, v ~ 5 N(0, I_3) (redrawn if a cell Peclet
               number |v_d| h_d / 2 reaches 1), t = 10^U(-3, 0), p uniform in {1..16}, m = 10,
               mixed precision (batched3d_instances)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20140707

WORKLOADS = {
    "tridiag-1d": dict(sides=(2000,), diff=1.0, vel=(0.0,), t=(1.0,), p=4, m=10, tol=1e-10,
                       seed=SEED_BASE + 1),
    "cd2d-256": dict(sides=(256, 256), diff=0.1, vel=(1.0, 1.0), t=(1e-3, 1e-2, 1e-1), p=8, m=10,
                     tol=1e-10, seed=SEED_BASE + 2),
    "toeplitz-1m": dict(n=1 << 20, bw=256, c=0.0, t=(1.0,), p=16, m=10, tol=1e-13,
                        seed=SEED_BASE + 3),
    "batched3d-64": dict(count=64, m=10, tol=1e-10, seed=SEED_BASE + 4),
    # one instance of the batched workload's largest class (96^3 grid, p = 16), for profiling
    "cd3d-96": dict(sides=(96, 96, 96), diff=1.0, vel=(1.0, -1.0, 0.5), t=(0.01,), p=16, m=10, tol=1e-10,
                    seed=SEED_BASE + 7),
    # a general sparse operator of the same size: the 96^3 grid's 7-point pattern with random
    # values (sparse_stencil_matrix), p = 16, for the sparse product and the inexact inverse
    "csr3d-96": dict(csr_sides=(96, 96, 96), t=(0.2,), p=16, m=10, tol=1e-10, seed=SEED_BASE + 11),
    # the large-norm Toeplitz regime of Example 5.4 (||A|| ~ 2e10 at n = 2^17): beta = 1.8,
    # p = 2, m = 30 and k = 30 deflated Ritz vectors as in the paper; t = 0.01 (at the paper's
    # t = 1 the result is ~1e-13 ||B||, below the CF approximation's own error), tol 1e-10
    "toeplitz-frac": dict(n=1 << 17, bw=(1 << 17) - 1, frac=1.8, d=2.0, t=(0.01,), p=2, m=30, k_defl=30,
                          tol=1e-10, seed=SEED_BASE + 6),
    # differentiation: L = ||r(tA) B - Y||_F^2, Y = r(t0 A) B0 (t0, B0 seeded perturbations)
    "cd2d-512-grad": dict(sides=(512, 512), diff=0.1, vel=(1.0, 1.0), t=(1e-2,), p=32, m=10,
                          tol=1e-10, seed=SEED_BASE + 5),
}


def batched3d_instances(count=64, seed=SEED_BASE + 4):
    """The seeded instance list of the batched workload: dicts with sides, diff (1), vel, t, p
    and the seed of the instance's right-hand side."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < count:
        sides = tuple(int(x) for x in rng.integers(32, 97, size=3))
        vel = tuple(float(x) for x in 5.0 * rng.standard_normal(3))
        t = float(10.0 ** rng.uniform(-3.0, 0.0))
        p = int(rng.integers(1, 17))
        if any(abs(v) / (2.0 * (N + 1)) >= 1.0 for v, N in zip(vel, sides)):
            continue
        out.append(dict(sides=sides, diff=1.0, vel=vel, t=t, p=p, seed=seed + 1000 + len(out)))
    return out


def toeplitz_column(bw, c=0.0):
    """First column (a_0, .., a_bw) of the Toeplitz workload: a_0 = -2 - c, a_k = 1/(1+k)^2."""
    a = np.empty(bw + 1)
    a[0] = -2.0 - c
    k = np.arange(1, bw + 1)
    a[1:] = 1.0 / (1.0 + k) ** 2
    return a


def fractional_column(n, beta=1.8, d=2.0):
    """First column of the symmetric Toeplitz operator of the large-norm workload: the
    symmetric part of Example 5.4's matrix.  The fractional diffusion equation there, with
    d_1 = 1 (left-sided) and d_2 = 3 (right-sided) derivatives of order beta and zero
    boundary values, discretised by the shifted Grunwald formula on h = 1/(n+1), gives
    A = (d_1 G + d_2 G^T) / h^beta with G the lower Hessenberg Toeplitz matrix
    G[i, j] = g_{i-j+1} (j <= i+1), g_k = (-1)^k binom(beta, k).  Its symmetric part is
    (d / h^beta)(G + G^T) with d = (d_1 + d_2) / 2 = 2: first column
    a_0 = 2 d g_1 / h^beta, a_1 = d (g_0 + g_2) / h^beta, a_k = d g_{k+1} / h^beta (k >= 2).
    The weights follow g_0 = 1, g_k = g_{k-1} (1 - (beta + 1) / k)."""
    g = np.empty(n + 1)
    g[0] = 1.0
    for k in range(1, n + 1):
        g[k] = g[k - 1] * (1.0 - (beta + 1.0) / k)
    scale = d * float(n + 1) ** beta
    a = np.empty(n)
    a[0] = 2.0 * g[1]
    if n > 1:
        a[1] = g[0] + g[2]
    a[2:] = g[3:n + 1]
    return scale * a


def grad_target(n, p, seed, t):
    """(t0, B0) of the differentiation workload: t0 = t (1 + 0.05 N(0,1)) (kept > 0),
    B0 = B + 0.1 N(0,1); B itself is rhs(n, p, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    t0 = max(1e-6, t * (1.0 + 0.05 * rng.standard_normal()))
    B0 = rhs(n, p, seed) + 0.1 * np.asfortranarray(rng.standard_normal((p, n)).T)
    return t0, B0


def sparse_dd_matrix(n, nnz_row=8, seed=SEED_BASE + 9, margin=(0.05, 0.5), scale=1.0e4):
    """A seeded nonsymmetric sparse n x n matrix for the general sparse operator: nnz_row - 1
    off-diagonal entries per row at random columns (N(0, 1) values), and a negative diagonal
    exceeding the row's off-diagonal magnitude by a factor 1 + U(margin), all times `scale`
    (rows weakly diagonally dominant with a negative diagonal, the operator's contract).
    Returns (indptr, indices, data) of the CSR form, column indices sorted within a row."""
    import numpy as np
    rng = np.random.default_rng(seed)
    k = max(0, nnz_row - 1)
    rows, cols, vals = [], [], []
    for i in range(n):
        js = rng.choice(n - 1, size=min(k, n - 1), replace=False)
        js = np.where(js >= i, js + 1, js)                      # off-diagonal columns
        v = rng.standard_normal(len(js))
        d = -(np.abs(v).sum() + 1e-3) * (1.0 + rng.uniform(*margin))
        js = np.concatenate([js, [i]])
        v = np.concatenate([v, [d]])
        order = np.argsort(js)
        rows.append(np.full(len(js), i))
        cols.append(js[order])
        vals.append(v[order] * scale)
    indices = np.concatenate(cols).astype(np.int32)
    data = np.concatenate(vals)
    indptr = np.zeros(n + 1, dtype=np.int64)
    indptr[1:] = np.cumsum([len(c) for c in cols])
    return indptr, indices, data


def sparse_stencil_matrix(sides, seed=SEED_BASE + 10, margin=(0.05, 0.5)):
    """A seeded sparse matrix with the 2-D/3-D grid's 5/7-point pattern (neighbours along each
    axis, x fastest, no wrap-around) but random N(0, 1) off-diagonal values, and a negative
    diagonal exceeding the row's off-diagonal magnitude by a factor 1 + U(margin) (rows weakly
    diagonally dominant with a negative diagonal, the general sparse operator's contract).
    Returns (indptr, indices, data) of the CSR form, columns sorted within a row."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sides = tuple(int(s_) for s_ in sides)
    n = int(np.prod(sides))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for s_ in sides:
        coords.append(rem % s_)
        rem //= s_
    rows, cols = [], []
    stride = 1
    for d, s_ in enumerate(sides):
        for sgn in (-1, 1):
            ok = (coords[d] + sgn >= 0) & (coords[d] + sgn < s_)
            rows.append(idx[ok])
            cols.append(idx[ok] + sgn * stride)
        stride *= s_
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = rng.standard_normal(len(r))
    off = np.bincount(r, weights=np.abs(v), minlength=n)
    dg = -(off + 1e-3) * (1.0 + rng.uniform(*margin, size=n))
    r = np.concatenate([r, idx])
    c = np.concatenate([c, idx])
    v = np.concatenate([v, dg])
    order = np.lexsort((c, r))
    indptr = np.zeros(n + 1, dtype=np.int64)
    indptr[1:] = np.cumsum(np.bincount(r, minlength=n))
    return indptr, c[order].astype(np.int32), v[order]


def rhs(n, p, seed):
    """B (n x p), i.i.d. N(0, 1), returned as a Fortran-ordered (column-major) array."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((p, n)).T)


def to_device_colmajor(B_np, device="cuda"):
    """Copy a numpy (n, p) array to a column-major (stride (1, n)) CUDA float64 tensor."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(B_np.T)).to(device).T
