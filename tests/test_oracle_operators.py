"""Pins for the oracle's operators and closed forms.

The sparse A (built from the stencil's Kronecker-sum definition) and the closed-form
eigen-expansion (diagonal similarity + DST-I) are written independently in
oracle/operators.py; here they are checked against each other, against a brute-force
stencil assembled point by point, against the textbook 1-D Laplacian eigenvalues
-4 (n+1)^2 sin^2(k pi / (2(n+1))), and against scipy's dense expm (the paper's own
'exact' solution method, Section 5).
"""
import numpy as np
import scipy.linalg as sl
import pytest

from oracle import operators as ops


def brute_force_stencil(sides, diff, vel, t):
    """Assemble t (diff Lap_h - v . grad_h) point by point (x fastest, Dirichlet 0)."""
    sides = list(sides)
    dims = len(sides)
    n = int(np.prod(sides))
    A = np.zeros((n, n))
    strides = [int(np.prod(sides[:d])) for d in range(dims)]
    for idx in range(n):
        coord = [(idx // strides[d]) % sides[d] for d in range(dims)]
        for d in range(dims):
            h = 1.0 / (sides[d] + 1)
            A[idx, idx] += t * (-2 * diff / h**2)
            for step, coef in ((-1, diff / h**2 + vel[d] / (2 * h)),
                               (+1, diff / h**2 - vel[d] / (2 * h))):
                c = coord[d] + step
                if 0 <= c < sides[d]:
                    A[idx, idx + step * strides[d]] += t * coef
    return A


CASES = [((9,), 1.0, (0.0,), 1.0), ((7, 6), 0.1, (1.0, 1.0), 0.05),
         ((5, 4, 3), 1.0, (2.0, -3.0, 1.5), 0.2), ((8, 5), 0.1, (-1.0, 0.5), 1.0)]


@pytest.mark.parametrize("sides,diff,vel,t", CASES)
def test_sparse_matches_brute_force(sides, diff, vel, t):
    A = ops.cd_matrix(sides, diff, vel, t).toarray()
    assert np.allclose(A, brute_force_stencil(sides, diff, vel, t), rtol=0, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("sides,diff,vel,t", CASES)
def test_closed_form_eigenpairs(sides, diff, vel, t):
    A = ops.cd_matrix(sides, diff, vel, t).toarray()
    lam = ops.eigenvalues(sides, diff, vel, t).ravel()
    ev = np.sort(np.linalg.eigvals(A).real)
    assert np.allclose(np.sort(lam), ev, rtol=1e-10, atol=1e-10 * np.abs(ev).max())
    assert np.all(lam < 0)                       # negative definite (Section 1)
    # f(A) B with f = identity reproduces A B
    rng = np.random.default_rng(3)
    B = rng.standard_normal((A.shape[0], 2))
    AB = ops.apply_function(sides, diff, vel, t, lambda l: l, B)
    assert np.allclose(AB, A @ B, rtol=1e-10, atol=1e-10 * np.abs(A @ B).max())


def test_textbook_1d_laplacian():
    n = 2000
    lam, _, _ = ops.axis_eig(n, 1.0, 0.0, 1.0)
    k = np.arange(1, n + 1)
    ref = -4.0 * (n + 1) ** 2 * np.sin(k * np.pi / (2 * (n + 1))) ** 2
    assert np.allclose(lam, ref, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("sides,diff,vel,t", CASES)
def test_closed_form_expm_vs_dense(sides, diff, vel, t):
    A = ops.cd_matrix(sides, diff, vel, t).toarray()
    rng = np.random.default_rng(5)
    B = rng.standard_normal((A.shape[0], 3))
    ref = sl.expm(A) @ B
    got = ops.exact_expm_B(sides, diff, vel, t, B)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def test_workload_operators_are_negative_definite_and_diag_similar():
    # 256x256, diff 0.1, v = (1,1): cell Peclet 1/(257*0.2) < 1 for every t
    for t in (1e-3, 1e-2, 1e-1):
        for N in (256, 512):
            lam, dp, _ = ops.axis_eig(N, 0.1, 1.0, t)
            assert np.all(lam < 0) and np.all(np.isfinite(dp))
