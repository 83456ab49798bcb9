"""Symmetric Toeplitz operators -- ORACLE (test infrastructure only; see oracle/__init__.py).

The paper's Example 5.4 (Section 5) applies the method to a Toeplitz matrix A, with products
computed by fast Toeplitz matrix-vector products (a 2n x 2n circulant embedding and FFTs, the
commented remark of Section 2) and the products with A^{-1} by the Gohberg-Semencul formula
(Section 4.1, where the inner solve is discussed; Example 5.4).  Here:
  - products: scipy's FFT-based Toeplitz product (a library primitive), dense on small n;
  - the exact inverse: the Gohberg-Semencul formula with the generator x = T^{-1} e_1 from
    the Levinson recursion (scipy.linalg.solve_toeplitz);
  - the truth for e^{tA} B: the Taylor series (||tA|| is small for the workload).

Workload (reading c = 0): first column a_0 = -2, a_k = 1/(1+k)^2 for 1 <= k <= 256, 0 beyond.
Its symbol a_0 + 2 sum_k a_k cos(k theta) lies in [-2.3551, -0.7179], so A is symmetric
negative definite.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def workload_column(n, bw=256, c=0.0):
    a = np.zeros(n)
    a[0] = -2.0 - c
    k = np.arange(1, min(bw, n - 1) + 1)
    a[k] = 1.0 / (1.0 + k) ** 2
    return a


def dense(a):
    return sl.toeplitz(a)


def matvec(a, V, t=1.0):
    """t T V for the symmetric Toeplitz T with first column a (scipy FFT product)."""
    V = np.asarray(V, dtype=np.float64)
    return t * sl.matmul_toeplitz((a, a), V, check_finite=False)


def symbol(a, theta):
    """f(theta) = a_0 + 2 sum_{k>=1} a_k cos(k theta), the generating function of T."""
    th = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    k = np.arange(1, len(a))
    return a[0] + 2.0 * np.cos(np.outer(th, k)) @ a[1:]


def symbol_range(a):
    """min / max of the symbol on a fine grid (bounds of the spectrum of every section)."""
    f = symbol(a, np.linspace(0, np.pi, 8193))
    return f.min(), f.max()


def taylor_expm_B(a, B, t=1.0, terms=60):
    """e^{tT} B by its Taylor series (converges fast: ||tT|| <= 2.36 for the workload)."""
    B = np.asarray(B, dtype=np.float64)
    term = B.copy()
    acc = B.copy()
    for j in range(1, terms + 1):
        term = matvec(a, term, t) / j
        acc += term
        if np.linalg.norm(term) <= 1e-20 * np.linalg.norm(acc):
            break
    return acc


# --------------------------------------------------------------------------- exact inverse
def lower_toeplitz_matvec(x, V, transpose=False):
    """L(x) V (or L(x)^T V) for the lower-triangular Toeplitz L(x) with first column x."""
    z = np.zeros_like(x)
    z[0] = x[0]
    if transpose:
        return sl.matmul_toeplitz((z, x), V, check_finite=False)
    return sl.matmul_toeplitz((x, z), V, check_finite=False)


def gsf_generator(a):
    """x = T^{-1} e_1 by the Levinson recursion (scipy.linalg.solve_toeplitz)."""
    e1 = np.zeros(len(a))
    e1[0] = 1.0
    return sl.solve_toeplitz((a, a), e1, check_finite=False)


def gsf_apply(x, V, t=1.0):
    """(tT)^{-1} V by the Gohberg-Semencul formula for symmetric Toeplitz T (Section 4.1;
    Example 5.4): with x = T^{-1} e_1 and xh = (0, x_{n-1}, ..., x_1),
        T^{-1} = ( L(x) L(x)^T - L(xh) L(xh)^T ) / x_0."""
    V = np.asarray(V, dtype=np.float64)
    xh = np.concatenate([[0.0], x[:0:-1]])
    u1 = lower_toeplitz_matvec(x, lower_toeplitz_matvec(x, V, transpose=True))
    u2 = lower_toeplitz_matvec(xh, lower_toeplitz_matvec(xh, V, transpose=True))
    return (u1 - u2) / (t * x[0])


# --------------------------------------------------------------------------- large-norm regime
def eig_function(a, B, f, t=1.0):
    """f(tT) B for the symmetric Toeplitz T with first column a, by the eigendecomposition
    T = Q diag(lambda) Q^T (scipy eigh; small n only): the exact truth where the Taylor series
    does not converge (||tT|| ~ 1e9 in Example 5.4's regime).  f maps an eigenvalue array to an
    array of the same shape."""
    lam, Q = sl.eigh(sl.toeplitz(a))
    B = np.asarray(B, dtype=np.float64)
    return Q @ (np.asarray(f(t * lam))[:, None] * (Q.T @ B))
