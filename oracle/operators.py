"""Test operators and their closed forms -- ORACLE (test infrastructure only).

The paper's problem (Section 1, eq. (1)): Z = e^{tA} B with tA large, sparse and negative
definite, t folded into A.  The workloads are constant-coefficient convection-diffusion
operators on the unit interval / square / cube with homogeneous Dirichlet boundaries
(the paper's Example 5.1 uses the 5-point Laplacian, a special case), discretised by
second-order central differences on N_d interior points per axis, h_d = 1/(N_d + 1):

    A = t * ( diff * Laplacian_h  -  v . grad_h )

Along one axis the 1-D factor is the tridiagonal Toeplitz matrix
    T = tridiag(l, c, u),  l = diff/h^2 + v/(2h),  c = -2 diff/h^2,  u = diff/h^2 - v/(2h)
(l multiplies u_{j-1}, u multiplies u_{j+1}), and A is the Kronecker sum of the axes'
factors, x fastest:  A = t (I_z (x) I_y (x) T_x + I_z (x) T_y (x) I_x + T_z (x) I_y (x) I_x).

Closed form used for the exact truths.  When l u > 0 (cell Peclet |v| h / (2 diff) < 1)
T = D^{-1} S D with D = diag(rho^j), rho = sqrt(u/l), and S = tridiag(s, c, s) symmetric,
s = sqrt(l u).  S = Q Lambda Q with the orthonormal DST-I matrix
    Q[j, k] = sqrt(2/(N+1)) sin(pi (j+1)(k+1)/(N+1)),  Lambda_k = c + 2 s cos(pi (k+1)/(N+1)).
So f(A) B = (x)_d (D_d^{-1} Q_d) . diag(f(t sum_d Lambda_d)) . (x)_d (Q_d D_d) . B.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tridiag_coeffs(N, diff, v, t=1.0):
    """(l, c, u) of t * (diff * d2/dx2 - v d/dx) on N interior points, h = 1/(N+1)."""
    h = 1.0 / (N + 1)
    l = diff / h**2 + v / (2 * h)
    c = -2.0 * diff / h**2
    u = diff / h**2 - v / (2 * h)
    return t * l, t * c, t * u


def axis_matrix(N, diff, v, t=1.0):
    l, c, u = tridiag_coeffs(N, diff, v, t)
    return sp.diags([np.full(N - 1, l), np.full(N, c), np.full(N - 1, u)], [-1, 0, 1],
                    format="csr")


def cd_matrix(sides, diff, vel, t=1.0):
    """The sparse A (CSR, FP64) for grid sides (N_x[, N_y[, N_z]]), x fastest."""
    sides = tuple(int(s) for s in sides)
    vel = tuple(float(v) for v in vel)
    A = None
    for d, N in enumerate(sides):
        T = axis_matrix(N, diff, vel[d], t)
        left = 1
        for e in range(d + 1, len(sides)):
            left *= sides[e]
        right = 1
        for e in range(d):
            right *= sides[e]
        term = sp.kron(sp.identity(left), sp.kron(T, sp.identity(right)))
        A = term if A is None else A + term
    return A.tocsr()


def axis_eig(N, diff, v, t=1.0):
    """Closed-form eigen-data of one axis factor: (lambda_k, rho_pow_j, Q)."""
    l, c, u = tridiag_coeffs(N, diff, v, t)
    if l * u <= 0:
        raise ValueError("cell Peclet number >= 1: axis factor not diagonally similar to "
                         "a symmetric matrix")
    s = np.sqrt(l * u) * np.sign(l)
    rho = np.sqrt(u / l)
    j = np.arange(N)
    k = np.arange(1, N + 1)
    lam = c + 2.0 * s * np.cos(np.pi * k / (N + 1))
    Q = np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * np.outer(j + 1, k) / (N + 1))
    return lam, rho ** j, Q


def _apply_axis(Xg, M, axis):
    """Multiply the tensor Xg (shape (..., N_axis, ...)) by M along ``axis``."""
    return np.moveaxis(np.tensordot(M, Xg, axes=([1], [axis])), 0, axis)


def eigenvalues(sides, diff, vel, t=1.0):
    """All eigenvalues of A as an array shaped like the grid (z, y, x order reversed)."""
    lam = None
    for d, N in enumerate(sides):
        ld, _, _ = axis_eig(N, diff, vel[d], t)
        shape = [1] * len(sides)
        shape[len(sides) - 1 - d] = N
        ld = ld.reshape(shape)
        lam = ld if lam is None else lam + ld
    return lam


def apply_function(sides, diff, vel, t, f, B):
    """f(A) B by the closed-form eigen-expansion; ``f`` maps an eigenvalue array to an
    array of the same shape (it may return np.longdouble / complex values).

    B is (n, p) with the grid index x fastest.  Transforms run in FP64; f is applied in
    whatever precision ``f`` returns, then rounded to FP64 before the inverse transform.
    """
    sides = tuple(int(s) for s in sides)
    dims = len(sides)
    p = B.shape[1]
    grid_shape = tuple(reversed(sides))          # (z, y, x) for C-order reshape
    X = np.asarray(B, dtype=np.float64).T.reshape((p,) + grid_shape)
    eig = []
    for d, N in enumerate(sides):
        eig.append(axis_eig(N, diff, vel[d], t))
    # forward: multiply by Q_d D_d along each axis
    for d in range(dims):
        lam, dpow, Q = eig[d]
        ax = 1 + (dims - 1 - d)
        X = _apply_axis(X, Q * dpow[None, :], ax)
    lam_all = eigenvalues(sides, diff, vel, t)
    fl = f(lam_all)
    X = (X * np.asarray(fl, dtype=np.float64)[None, ...]) if not np.iscomplexobj(fl) else \
        (X * np.asarray(fl)[None, ...])
    # inverse: multiply by D_d^{-1} Q_d along each axis
    for d in range(dims):
        lam, dpow, Q = eig[d]
        ax = 1 + (dims - 1 - d)
        X = _apply_axis(X, Q / dpow[:, None], ax)
    return np.ascontiguousarray(X.reshape(p, -1).T)


def r_of_lambda_ext(table, lam):
    """r(lambda) = omega_0 + sum 2 Re(omega_i/(lambda - tau_i)) in extended precision.

    The partial-fraction sum cancels badly where r is small (r(lambda) ~ e^lambda while
    the terms are ~|omega_i|/|tau_i|), so the exact truth evaluates it in np.longdouble
    from the FP64 table values, then rounds the result to FP64.
    """
    L = np.asarray(lam, dtype=np.longdouble)
    r = np.full(L.shape, np.longdouble(table["omega0"]))
    for tau, om in zip(table["tau"], table["omega"]):
        tr, ti = np.longdouble(tau.real), np.longdouble(tau.imag)
        orr, oi = np.longdouble(om.real), np.longdouble(om.imag)
        dr = L - tr
        den = dr * dr + ti * ti
        # omega / (lambda - tau) = omega * conj(lambda - tau) / |lambda - tau|^2
        # lambda - tau = dr - i ti ; conj = dr + i ti
        re = (orr * dr - oi * ti) / den
        r = r + 2 * re
    return r.astype(np.float64)


def exact_r_of_A_B(sides, diff, vel, t, table, B):
    """The method's exact target r(A) B (closed form, r evaluated in extended precision)."""
    return apply_function(sides, diff, vel, t, lambda lam: r_of_lambda_ext(table, lam), B)


def exact_expm_B(sides, diff, vel, t, B):
    """e^{A} B by the closed form (the paper's quantity of interest, eq. (1))."""
    return apply_function(sides, diff, vel, t, np.exp, B)
