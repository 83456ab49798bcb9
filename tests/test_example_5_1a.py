"""Replay of the paper's Example 5.1a (Section 5, Table 5.1) with the oracle.

The matrix -2500 gallery('poisson', 99) is t * diff * Laplacian_h on a 99 x 99 grid with
diff = 0.25 (since (99+1)^2 = 1e4), B = randn(9801, 3), m = 30, tol = 1e-8.  Table 5.1 prints
Mat-Vec 123 for PSBFOM-DR and 810 for SBFOM-DR (k = 30).  Pinned here: the preconditioned
algorithm converges within the paper's Mat-Vec count and within its error, and needs several
times fewer Mat-Vecs than the unpreconditioned one (the paper's ratio is 810/123 = 6.6).
"""
import json
import os

import numpy as np
import pytest

from oracle import cf, operators as ops, psbfom as ps

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_5_1.json")))


@pytest.mark.slow
def test_example_5_1a_matvec_counts():
    tab = cf.load_table()
    sides, diff, vel, t = (99, 99), 0.25, (0.0, 0.0), 1.0
    A = ops.cd_matrix(sides, diff, vel, t)
    assert A.diagonal()[0] == -10000.0 and A[0, 1] == 2500.0      # -2500 * poisson(99)
    B = np.random.default_rng(2014).standard_normal((9801, 3))
    ex = ops.exact_expm_B(sides, diff, vel, t, B)
    Z2, i2 = ps.psbfom(ps.lu_inverse(A), B, tab, m=30, tol=1e-8, max_cycles=50, k=30)
    Z1, i1 = ps.sbfom(ps.matvec(A), B, tab, m=30, tol=1e-8, max_cycles=2000)
    assert i2["converged"] and i1["converged"]
    e2 = np.linalg.norm(Z2 - ex) / np.linalg.norm(ex)
    e1 = np.linalg.norm(Z1 - ex) / np.linalg.norm(ex)
    assert i2["matvecs"] <= GOLD["psbfom_dr"]["matvec"]
    assert e2 <= GOLD["psbfom_dr"]["error"] and e1 <= 10 * GOLD["sbfom_dr"]["error"]
    assert i1["matvecs"] >= 6 * i2["matvecs"]
