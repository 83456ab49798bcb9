"""Pins of the symmetric Toeplitz oracle (Example 5.4) against facts outside itself.

- the symbol's extreme values from the closed sums pi^2/6 and pi^2/12 (not the oracle's grid);
- products against an explicit double loop (brute force);
- Taylor truth against scipy's Pade expm on a dense matrix (a different algorithm);
- the Gohberg-Semencul inverse against a dense solve;
- Algorithm 1 and Algorithm 2 of the oracle on a Toeplitz operator against the Taylor truth.
Each pin fails under a planted mistake (last test).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import cf, psbfom, toeplitz as TZ


def test_symbol_closed_form():
    from scipy.special import polygamma
    a = TZ.workload_column(4096)
    # f(0) = -2 + 2 sum_{j=2}^{257} 1/j^2 and f(pi) = -2 + 2 sum_{j=2}^{257} (-1)^{j-1}/j^2, from
    # pi^2/6, pi^2/12 and the trigamma tails sum_{j>=N} 1/j^2 = psi'(N)
    tail = polygamma(1, 258)
    alt_tail = 0.25 * (polygamma(1, 129.5) - polygamma(1, 129))   # sum_{j>=258} (-1)^{j-1}/j^2
    f0 = -2.0 + 2.0 * (math.pi ** 2 / 6 - 1.0 - tail)
    fpi = -2.0 + 2.0 * (math.pi ** 2 / 12 - 1.0 - alt_tail)
    assert abs(TZ.symbol(a, 0.0)[0] - f0) < 1e-13 and abs(TZ.symbol(a, math.pi)[0] - fpi) < 1e-13
    lo, hi = TZ.symbol_range(a)
    assert abs(hi - f0) < 1e-13                    # the maximum is at theta = 0 (all a_k > 0)
    assert fpi - 1e-4 < lo <= fpi                  # the truncation ripple dips just below f(pi)
    assert -2.3552 < lo < -2.3550 and -0.7180 < hi < -0.7178


def test_eigenvalues_inside_symbol_range():
    a = TZ.workload_column(600)
    lo, hi = TZ.symbol_range(a)
    ev = np.linalg.eigvalsh(TZ.dense(a))
    assert ev.min() >= lo - 1e-12 and ev.max() <= hi + 1e-12


@pytest.mark.parametrize("n,bw", [(37, 256), (300, 256), (300, 17)])
def test_matvec_brute_force(n, bw):
    a = TZ.workload_column(n, bw=bw)
    V = np.random.default_rng(n + bw).standard_normal((n, 3))
    W = np.zeros_like(V)
    for i in range(n):
        for j in range(n):
            W[i] += a[abs(i - j)] * V[j]
    assert np.abs(TZ.matvec(a, V, 0.7) - 0.7 * W).max() < 1e-13


def test_taylor_vs_pade():
    a = TZ.workload_column(200)
    B = np.random.default_rng(3).standard_normal((200, 4))
    ref = sl.expm(TZ.dense(a)) @ B
    Z = TZ.taylor_expm_B(a, B, 1.0)
    assert np.linalg.norm(Z - ref) / np.linalg.norm(ref) < 1e-14


@pytest.mark.parametrize("n,bw,t", [(64, 256, 1.0), (257, 40, 0.5), (500, 256, 2.0)])
def test_gsf_inverse(n, bw, t):
    a = TZ.workload_column(n, bw=bw)
    x = TZ.gsf_generator(a)
    assert np.abs(TZ.dense(a) @ x - np.eye(n)[:, 0]).max() < 1e-14
    V = np.random.default_rng(n).standard_normal((n, 3))
    W = TZ.gsf_apply(x, V, t)
    ref = np.linalg.solve(t * TZ.dense(a), V)
    assert np.linalg.norm(W - ref) / np.linalg.norm(ref) < 1e-14


@pytest.fixture(scope="module")
def table():
    return cf.load_table()


def test_sbfom_and_psbfom_on_toeplitz(table):
    n, p = 3000, 4
    a = TZ.workload_column(n)
    B = np.random.default_rng(11).standard_normal((n, p))
    truth = TZ.taylor_expm_B(a, B, 1.0)
    tol = 1e-13
    Z1, i1 = psbfom.sbfom(lambda W: TZ.matvec(a, W), B, table, m=10, tol=tol)
    x = TZ.gsf_generator(a)
    Z2, i2 = psbfom.psbfom(lambda W: TZ.gsf_apply(x, W), B, table, m=10, tol=tol)
    assert i1["converged"] and i2["converged"]
    # CF error (max |r - exp| on (-inf, 0]) plus the solver's share: the residual split of
    # error analysis of Section 4.2, sum_i |omega_i| ||(A - tau_i I)^{-1}|| rho_i, rho_i <= tol ||B||
    lo, hi = TZ.symbol_range(a)
    dist = [abs(complex(min(max(t.real, lo), hi), 0.0) - t) for t in table["tau"]]
    solver = sum(abs(w) / d for w, d in zip(table["omega"], dist)) * tol
    bound = (1.1 * table["sigma"] + solver) * np.linalg.norm(B) / np.linalg.norm(truth)
    for Z in (Z1, Z2):
        assert np.linalg.norm(Z - truth) / np.linalg.norm(truth) < bound


def test_planted_mistakes_fail():
    """A dropped term, a wrong sign and a transposed factor each break a pin above."""
    n = 120
    a = TZ.workload_column(n, bw=30)
    V = np.random.default_rng(5).standard_normal((n, 2))
    ref_inv = np.linalg.solve(TZ.dense(a), V)
    x = TZ.gsf_generator(a)
    xh = np.concatenate([[0.0], x[:0:-1]])
    # dropped second term of the formula
    W = TZ.lower_toeplitz_matvec(x, TZ.lower_toeplitz_matvec(x, V, transpose=True)) / x[0]
    assert np.linalg.norm(W - ref_inv) > 1e-3 * np.linalg.norm(ref_inv)
    # wrong sign between the terms
    W = (TZ.lower_toeplitz_matvec(x, TZ.lower_toeplitz_matvec(x, V, transpose=True))
         + TZ.lower_toeplitz_matvec(xh, TZ.lower_toeplitz_matvec(xh, V, transpose=True))) / x[0]
    assert np.linalg.norm(W - ref_inv) > 1e-3 * np.linalg.norm(ref_inv)
    # transposed inner factor
    W = (TZ.lower_toeplitz_matvec(x, TZ.lower_toeplitz_matvec(x, V))
         - TZ.lower_toeplitz_matvec(xh, TZ.lower_toeplitz_matvec(xh, V))) / x[0]
    assert np.linalg.norm(W - ref_inv) > 1e-3 * np.linalg.norm(ref_inv)
    # a product that drops the symmetric half (lower triangle only)
    Wl = sl.matmul_toeplitz((a, np.r_[a[0], np.zeros(n - 1)]), V)
    assert np.abs(Wl - TZ.matvec(a, V)).max() > 1e-3


# --------------------------------------------------------------------------- Example 5.4 regime
def test_fractional_column_against_its_definition():
    """The large-norm workload's column (inputs.fractional_column) against the definition it
    states, built independently: g_k = (-1)^k binom(beta, k) from scipy's binomial, the shifted
    Grunwald matrix G[i, j] = g_{i-j+1} assembled entry by entry, A = (d / h^beta)(G + G^T)."""
    from scipy.special import binom
    from paper_1405_0707_gb300 import inputs
    n, beta, d = 200, 1.8, 2.0
    a = inputs.fractional_column(n, beta, d)
    g = np.array([(-1.0) ** k * binom(beta, k) for k in range(n + 2)])
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(min(n, i + 2)):
            G[i, j] = g[i - j + 1]
    A = d * (n + 1) ** beta * (G + G.T)
    assert np.allclose(TZ.dense(a), A, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    # (1 - 1)^beta = 0: the weights sum to zero; with g_1 = -beta the others sum to beta
    assert abs(g[0] + g[2:].sum() - beta) < 0.05 and abs(g[1] + beta) < 1e-15 and np.all(g[2:] > 0)


def test_fractional_operator_is_negative_definite_with_large_norm():
    """Negative definite (the symbol's largest value a_0 + 2 sum a_k is negative, and so are the
    eigenvalues of a section), with ||A|| of the order 1e9 at n = 5e4 and 1e10 at n = 2e5 as the
    paper states for its Example 5.4 matrices."""
    from paper_1405_0707_gb300 import inputs
    a = inputs.fractional_column(400)
    assert np.linalg.eigvalsh(TZ.dense(a)).max() < 0
    for n, lo, hi in ((50000, 1e9, 1e10), (200000, 1e10, 1e11)):
        a = inputs.fractional_column(n)
        norm_bound = abs(a[0]) + 2 * np.abs(a[1:]).sum()       # ||A||_1 = ||A||_inf >= ||A||_2
        assert lo <= norm_bound < hi, (n, norm_bound)
        assert a[0] + 2 * np.sort(a[1:])[::-1].sum() < 0


def test_eig_function_against_dense_solves_and_expm(table):
    """The eigendecomposition truth against the partial-fraction sum by dense solves (eq. (11))
    and against scipy's expm, on a fractional operator small enough for both."""
    from paper_1405_0707_gb300 import inputs
    from oracle import psbfom as ps
    a = inputs.fractional_column(300)
    B = np.random.default_rng(7).standard_normal((300, 2))
    t = 1e-3
    r_eig = TZ.eig_function(a, B, lambda lam: __import__("oracle.operators", fromlist=["x"]).r_of_lambda_ext(table, lam), t)
    r_dense = ps.dense_r_of_A_B(t * TZ.dense(a), B, table)
    assert np.linalg.norm(r_eig - r_dense) <= 1e-9 * np.linalg.norm(r_dense)
    e_eig = TZ.eig_function(a, B, np.exp, t)
    assert np.linalg.norm(e_eig - sl.expm(t * TZ.dense(a)) @ B) <= 1e-9 * np.linalg.norm(e_eig)


def test_gsf_on_a_large_norm_operator():
    """The Gohberg-Semencul inverse with the Levinson generator on a fractional operator
    (kappa ~ 1e6 at n = 1024): against a dense solve, to the conditioning limit."""
    from paper_1405_0707_gb300 import inputs
    a = inputs.fractional_column(1024)
    T = TZ.dense(a)
    V = np.random.default_rng(8).standard_normal((1024, 3))
    x = TZ.gsf_generator(a)
    got = TZ.gsf_apply(x, V, 1.0)
    ref = np.linalg.solve(T, V)
    kappa = np.linalg.cond(T)
    assert 1e5 < kappa < 1e8
    assert np.linalg.norm(got - ref) <= 1e-14 * kappa * np.linalg.norm(ref)
