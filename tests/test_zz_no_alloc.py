"""The allocation-free exact-inverse apply (expm_prec_apply_noalloc), through the C ABI.

Some callers cannot call cudaMalloc (their own pool allocator owns the device memory, or a
latency-critical loop must not enter the CUDA allocator); this entry point serves them with
a fixed scratch array inside the library instead of a plan.  Its output must match the
plan-based expm_prec_apply and the oracle's sparse LU solve on consecutive calls (each call
reuses the scratch that the one before filled, with a different operator and shape; the
1-D call follows a larger 2-D one).  Collected last on purpose.
"""
import numpy as np
import pytest

from paper_1405_0707_gb300 import inputs
from tests.gpu_util import need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _desc(sides, diff, vel):
    from paper_1405_0707_gb300 import _native as N
    op = N.expm_op_desc()
    op.kind, op.ndim, op.diff = N.EXPM_OP_CONV_DIFF, len(sides), float(diff)
    for d in range(3):
        op.side[d] = sides[d] if d < len(sides) else 1
        op.vel[d] = vel[d] if d < len(vel) else 0.0
    return op


def test_noalloc_matches_plan_apply_and_oracle_on_consecutive_calls():
    torch = need_gpu()
    from oracle import operators as ops, psbfom as ps
    from paper_1405_0707_gb300 import Plan, colmajor
    from paper_1405_0707_gb300 import _native as N
    # the 1-D call comes after a larger 2-D call has filled the scratch
    calls = [((256, 256), 0.1, (1.0, 1.0), 1e-1, 8), ((37, 29), 0.1, (1.0, -0.5), 1e-2, 3),
             ((2000,), 1.0, (0.0,), 1.0, 4)]
    for k, (sides, diff, vel, t, p) in enumerate(calls):
        n = int(np.prod(sides))
        Vh = inputs.rhs(n, p, 500 + k)
        V = to_dev(Vh)
        ref = to_np(Plan(sides, diff, vel, p_max=p, m=2).prec_apply(t, V))
        W = colmajor(n, p)
        W.fill_(float("nan"))
        stream = torch.cuda.current_stream().cuda_stream
        N.expm_prec_apply_noalloc(_desc(sides, diff, vel), t, V.data_ptr(), V.stride(1), p,
                                  W.data_ptr(), W.stride(1), stream)
        torch.cuda.synchronize()
        got = to_np(W)
        assert np.all(np.isfinite(got))
        assert rel(got, ref) <= 1e-13, (k, rel(got, ref))
        # against the oracle's sparse LU solve (the paper's "LU once and for all"); the
        # transform path's backward error grows with the diagonal similarity's condition
        # number along the transformed axis
        Ainv = ps.lu_inverse(ops.cd_matrix(sides, diff, vel, t))
        lu = np.column_stack([Ainv(Vh[:, c]) for c in range(p)])
        kappa = 1.0
        for d in range(1, len(sides)):
            _, dp, _ = ops.axis_eig(sides[d], diff, vel[d], t)
            kappa *= dp.max() / dp.min()
        assert rel(got, lu) <= 1e-13 * max(1.0, kappa) + 1e-13, (k, rel(got, lu))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = need_gpu()
    from paper_1405_0707_gb300 import colmajor
    from paper_1405_0707_gb300 import _native as N
    n, p = 512 * 512, 8                      # T1 alone needs n p = 2^21 doubles > 2^20
    V, W = colmajor(n, p), colmajor(n, p)
    with pytest.raises(N.ExpmError) as e:
        N.expm_prec_apply_noalloc(_desc((512, 512), 0.1, (1.0, 1.0)), 0.1, V.data_ptr(), n, p,
                                  W.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == N.EXPM_INVALID_ARG
