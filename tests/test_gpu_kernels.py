"""GPU parity of the hot-path kernels against the oracle, through the C ABI.

Sizes span several 16-row tiles, 64x64 GEMM tiles and ragged tails (n not a multiple of
16, 32 or 64), in 1-D, 2-D and 3-D.
"""
import numpy as np
import pytest

from oracle import operators as ops, psbfom as ps
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

CASES = [((517,), 1.0, (0.0,), 1.0, 3),
         ((37, 29), 0.1, (1.0, 1.0), 1e-2, 3),
         ((70, 66), 0.1, (1.0, -0.5), 1e-1, 5),
         ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.3, 2),
         ((256, 256), 0.1, (1.0, 1.0), 1e-2, 8)]


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES)
def test_op_apply_matches_sparse_matrix(sides, diff, vel, t, p):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    V = inputs.rhs(n, p, 1234)
    plan = Plan(sides, diff, vel, p_max=p, m=2)
    W = to_np(plan.op_apply(t, to_dev(V)))
    ref = ops.cd_matrix(sides, diff, vel, t) @ V
    assert np.max(np.abs(W - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES)
def test_prec_apply_matches_sparse_lu(sides, diff, vel, t, p):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    V = inputs.rhs(n, p, 99)
    plan = Plan(sides, diff, vel, p_max=p, m=2)
    W = to_np(plan.prec_apply(t, to_dev(V)))
    Ainv = ps.lu_inverse(ops.cd_matrix(sides, diff, vel, t))
    ref = np.column_stack([Ainv(V[:, c]) for c in range(p)])
    # exact solve in both; the transform path's backward error grows with the diagonal
    # similarity's condition number (rho^-N per transformed axis)
    kappa = 1.0
    for d in range(1, len(sides)):
        _, dp, _ = ops.axis_eig(sides[d], diff, vel[d], t)
        kappa *= dp.max() / dp.min()
    assert rel(W, ref) <= 1e-13 * max(1.0, kappa) + 1e-13
    # and A (A^{-1} V) = V through the independent sparse matrix
    A = ops.cd_matrix(sides, diff, vel, t)
    assert rel(A @ W, V) <= 1e-11 * max(1.0, kappa)


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES[:4])
def test_block_arnoldi_matches_ruhe_variant(sides, diff, vel, t, p):
    """Cholesky-QR blocks with a positive diagonal reproduce Ruhe's vector-wise basis
    (Section 3): V and H~ agree element by element with the oracle's."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    m = 4
    V1, _ = ps.qr_positive(inputs.rhs(n, p, 7))
    plan = Plan(sides, diff, vel, p_max=p, m=m)
    Vg, Hg = plan.arnoldi(t, to_dev(V1))
    Vg, Hg = to_np(Vg), to_np(Hg)
    Ainv = ps.lu_inverse(ops.cd_matrix(sides, diff, vel, t))
    Vo, Ho, m_done, bd = ps.block_arnoldi_ruhe(Ainv, V1, m)
    assert not bd
    assert np.max(np.abs(Hg - Ho)) <= 1e-9 * np.max(np.abs(Ho))
    assert np.max(np.abs(Vg - Vo)) <= 1e-8
    assert np.linalg.norm(Vg.T @ Vg - np.eye((m + 1) * p)) <= 1e-13 * (m + 1) * p
    # band upper Hessenberg with p sub-diagonals, H_{j+1,j} upper triangular
    assert np.all(Hg[np.tril_indices_from(Hg, -p - 1)] == 0.0)
