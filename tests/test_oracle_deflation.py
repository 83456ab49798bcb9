"""Pins for the oracle's deflated restart (the restart of Algorithm 1 with deflation, used by
Algorithm 2 with the Krylov operator A^{-1}; Remark 4.1 for which Ritz values to keep).

* The selection rule against matrices whose eigenvalues are known by construction (an
  orthogonal similarity of a block-diagonal matrix of real values and 2 x 2 rotation-scaling
  blocks): the kept count is a multiple of the block width, conjugate pairs are never split,
  span(P) is invariant under H, and the eigenvalues of P^T H P are exactly the wanted ones.
* After a deflated restart the block Arnoldi relation Op V_m = V_{m+1} H~_m still holds
  (a wrong projection of H~ onto the kept vectors breaks it).
* Both algorithms with deflation converge to the closed-form r(tA) B, in no more Mat-Vecs
  than without it.
"""
import numpy as np
import pytest

from oracle import cf, operators as ops, psbfom as ps


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def known_spectrum_matrix(reals, pairs, seed):
    """H = U D U^T with D = blkdiag(reals, [[a, b], [-b, a]] per pair a + ib); eigenvalues known."""
    n = len(reals) + 2 * len(pairs)
    D = np.zeros((n, n))
    i = 0
    for r in reals:
        D[i, i] = r
        i += 1
    for a, b in pairs:
        D[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
        i += 2
    U, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    lam = np.r_[np.asarray(reals, dtype=complex), [complex(a, b) for a, b in pairs],
                [complex(a, -b) for a, b in pairs]]
    return U @ D @ U.T, lam


def test_selection_rule_on_known_spectrum():
    # moduli: reals 9, 7, 3, 1; pairs |8+1i| = 8.06, |2+5i| = 5.39, |0.5+0.5i| = 0.71
    H, lam = known_spectrum_matrix([9.0, 7.0, 3.0, 1.0], [(8.0, 1.0), (2.0, 5.0), (0.5, 0.5)], 3)
    cases = [
        # (k, align, largest) -> wanted eigenvalue multiset
        ((3, 1, True), [9, complex(8, 1), complex(8, -1)]),
        ((2, 2, True), [9, 7]),                  # the pair 8+-i does not fit after 9 -> next real
        ((4, 2, True), [9, complex(8, 1), complex(8, -1), 7]),
        ((3, 3, True), [9, complex(8, 1), complex(8, -1)]),
        ((2, 1, False), [complex(0.5, 0.5), complex(0.5, -0.5)]),
        ((3, 3, False), [complex(0.5, 0.5), complex(0.5, -0.5), 1]),
        ((4, 4, False), [complex(0.5, 0.5), complex(0.5, -0.5), 1, 3]),
    ]
    for (k, align, largest), want in cases:
        P = ps.deflation_basis(H, k, largest, align=align)
        assert P.shape[1] % align == 0 and P.shape[1] == len(want), (k, align, largest, P.shape)
        assert np.allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-12)
        M = P.T @ H @ P
        assert np.linalg.norm(H @ P - P @ M) <= 1e-12 * np.linalg.norm(H)
        got = np.sort_complex(np.linalg.eigvals(M))
        assert np.allclose(got, np.sort_complex(np.asarray(want, dtype=complex)), atol=1e-10), (k, align, got)


def test_selection_drops_to_a_multiple_of_the_block_width():
    # only pairs: with align 3 and k 3 the first pair fits (2), the next does not (4 > 3) and
    # there is no real value, so the count 2 drops to 0 (no deflation this restart)
    H, _ = known_spectrum_matrix([], [(1.0, 2.0), (3.0, 1.0), (0.1, 4.0)], 5)
    assert ps.deflation_basis(H, 3, True, align=3).shape[1] == 0
    assert ps.deflation_basis(H, 4, True, align=2).shape[1] == 4


@pytest.mark.parametrize("alg", [1, 2])
def test_arnoldi_relation_holds_after_deflated_restart(tab, alg):
    sides, diff, vel, t = (20, 18), 0.1, (1.0, -1.0), (0.05 if alg == 1 else 1.0)
    A = ops.cd_matrix(sides, diff, vel, t)
    B = np.random.default_rng(21).standard_normal((A.shape[0], 3))
    op = ps.lu_inverse(A) if alg == 2 else ps.matvec(A)
    m, p, k = 5, 3, 6
    if alg == 2:
        _, info = ps.psbfom(op, B, tab, m=m, k=k, align=p, fixed_cycles=3, return_details=True)
        dets = info["details"]
    else:
        # Algorithm 1: re-run the restart by hand from the oracle's pieces
        V1, _ = ps.qr_positive(B)
        V, H, _, _ = ps.block_arnoldi_ruhe(op, V1, m)
        Pk = ps.deflation_basis(H[:m * p, :m * p], k, largest=False, align=p)
        kk = Pk.shape[1]
        Pk1 = np.zeros(((m + 1) * p, kk + p))
        Pk1[:m * p, :kk] = Pk
        Pk1[m * p:, kk:] = np.eye(p)
        Vn = V @ Pk1
        V2, H2, _, _ = ps.block_arnoldi_ruhe(op, Vn[:, kk:kk + p], m, Vn, Pk1.T @ H @ Pk)
        dets = [{"V": V, "H": H}, {"V": V2, "H": H2}]
    for d in dets[1:]:
        V, H = d["V"], d["H"]
        W = np.column_stack([op(V[:, c]) for c in range(m * p)])
        assert np.linalg.norm(W - V @ H) <= 1e-10 * np.linalg.norm(W)
        assert np.linalg.norm(V.T @ V - np.eye(V.shape[1])) <= 1e-12


def test_both_algorithms_with_deflation_match_closed_form(tab):
    sides, diff, vel = (24, 20), 0.1, (1.0, 1.0)
    B = np.random.default_rng(22).standard_normal((24 * 20, 3))
    for alg, t in ((2, 1.0), (1, 0.05)):
        A = ops.cd_matrix(sides, diff, vel, t)
        ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
        run = (lambda **kw: ps.psbfom(ps.lu_inverse(A), B, tab, **kw)) if alg == 2 else \
              (lambda **kw: ps.sbfom(ps.matvec(A), B, tab, **kw))
        Z0, i0 = run(m=5, tol=1e-12, max_cycles=400)
        Zk, ik = run(m=5, tol=1e-12, max_cycles=400, k=6, align=3)
        assert i0["converged"] and ik["converged"], alg
        assert rel(Z0, ref) < 1e-10 and rel(Zk, ref) < 1e-10, (alg, rel(Zk, ref))
        assert ik["matvecs"] <= i0["matvecs"], (alg, ik["matvecs"], i0["matvecs"])
