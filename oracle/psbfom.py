"""Shifted block FOM (Algorithm 1) and preconditioned shifted block FOM (Algorithm 2)
-- ORACLE (test infrastructure only; see oracle/__init__.py).

Written step by step in the paper's order and notation, in plain numpy/scipy FP64.
Nothing here is blocked, fused or reordered beyond what the paper states:

* block Arnoldi with A. Ruhe's variant (Section 3, eq. (2.1)): one new basis vector at
  a time, w = Op v_k orthogonalised against every earlier vector.  The oracle runs the
  Gram-Schmidt loop twice per vector (the second pass is a no-op in exact arithmetic and
  only keeps the computed basis orthonormal to working accuracy);
* Algorithm 2 (Section 4.1): Krylov operator A^{-1} (eq. (4.5)), projected systems
  (I - tau_i H_m) Z_i = E_1 R_i (eq. (3236)), residual norms |tau_i| ||H_{m+1,m} E_m^T Z_i||_F
  (eq. (49)), restart from V_{m+1} with the collinear residual factors, and, when the
  cycles stop, X_i = A^{-1} Y_i (text after eq. (3188)) and
  Z = omega_0 B + sum_i omega_i X_i (Section 4.2, error analysis; eq. (11));
* Algorithm 1 (Section 3): Krylov operator A, projected systems (H_m - tau_i I) Z_i = E_1 R_i
  (eq. (3.3)), residuals -V_{m+1} H_{m+1,m} E_m^T Z_i (eq. (35)), norms by eq. (365).

Conjugate poles: for real A and B, (A - conj(tau) I)^{-1} B = conj((A - tau I)^{-1} B), so
the oracle solves the nu/2 poles with Im tau > 0 and adds 2 Re(omega_i X_i) (Section 2,
last paragraph before Remark 2.1).

Readings of the paper where it is silent: stop when max_i ||R_i||_F <= tol ||B||_F;
a block Arnoldi breakdown (new vector norm <= 1e-14 of its norm before orthogonalisation)
ends the cycle; deflation (the deflated restart of Algorithms 1 and 2) is
``k`` > 0, Ritz values of H_m chosen as the k smallest in modulus for Algorithm 1 and the
k largest in modulus for Algorithm 2 (Remark 4.1: those are the smallest |lambda(A)|).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------- helpers
def lu_inverse(A):
    """A^{-1} by one sparse LU, then two triangular solves per product (Section 4.1,
    'LU factorization ... performed once and for all'; Section 5: [L,U] = lu(A),
    A^{-1} w = U \\ (L \\ w))."""
    lu = spla.splu(A.tocsc())

    def apply(w):
        return lu.solve(np.asarray(w, dtype=np.float64))
    return apply


def matvec(A):
    def apply(w):
        return A @ np.asarray(w, dtype=np.float64)
    return apply


def qr_positive(B):
    """The initial block QR of Algorithm 1: B = V_1 R with V_1 orthonormal, R upper triangular with a
    positive diagonal (Householder QR, then column signs fixed)."""
    Q, R = np.linalg.qr(B)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def block_arnoldi_ruhe(op, V1, m, start_vectors=None, H0=None):
    """Block Arnoldi, A. Ruhe's variant (Section 3, eq. (2.1)).

    Generates v_{p+1}, ..., v_{(m+1)p}: the vector v_j comes from w = op(v_{j-p}),
    orthogonalised against v_1..v_{j-1} (twice), h_{j,j-p} = ||w||, v_j = w / h.
    ``start_vectors``/``H0`` let a deflated restart continue from a given leading basis
    (the deflated restart of Algorithm 1): columns [0, len0) of the basis and the corresponding leading
    columns of H are taken as given.

    Returns (V, H, m_done, breakdown): V is n x (m_done+1)p, H is (m_done+1)p x m_done p.
    """
    n, p = V1.shape if start_vectors is None else (start_vectors.shape[0], V1.shape[1])
    V = np.zeros((n, (m + 1) * p), order="F")     # basis vectors are columns
    H = np.zeros(((m + 1) * p, m * p))
    if start_vectors is None:
        V[:, :p] = V1
        first = p
    else:
        first = start_vectors.shape[1]
        V[:, :first] = start_vectors
        H[:H0.shape[0], :H0.shape[1]] = H0
    breakdown = False
    m_done = m
    for j in range(first, (m + 1) * p):
        k = j - p
        w = op(V[:, k])
        norm0 = np.linalg.norm(w)
        for _ in range(2):
            for i in range(j):
                h = V[:, i] @ w
                w = w - h * V[:, i]
                H[i, k] += h
        hn = np.linalg.norm(w)
        if hn <= 1e-14 * max(norm0, 1e-300):
            # Breakdown (reading: the paper is silent).  Only the clean case is handled:
            # the first vector of a new block already lies in the span, and so do the
            # images of the block's other columns -> an invariant subspace; the cycle
            # ends with m_done = k/p + 1 blocks and H_{m_done+1, m_done} = 0.
            if k % p != 0:
                raise NotImplementedError("partial block breakdown inside a block")
            b = k // p
            for kk in range(k + 1, (b + 1) * p):
                w = op(V[:, kk])
                n0 = np.linalg.norm(w)
                for _ in range(2):
                    for i in range(j):
                        h = V[:, i] @ w
                        w = w - h * V[:, i]
                        H[i, kk] += h
                if np.linalg.norm(w) > 1e-12 * max(n0, 1e-300):
                    raise NotImplementedError("partial block breakdown")
            breakdown = True
            m_done = b + 1
            V[:, j:] = 0.0
            break
        H[j, k] = hn
        V[:, j] = w / hn
    if breakdown:
        V = V[:, :(m_done + 1) * p]
        H = H[:(m_done + 1) * p, :m_done * p]
    return V, H, m_done, breakdown


def deflation_basis(Hm, k, largest, align=None):
    """The eigenproblem of the deflated restart (Algorithm 1): eigenpairs of H_m; keep the k wanted ones (smallest |theta|
    for Algorithm 1, largest |theta| for Algorithm 2 -- Remark 4.1), split complex
    eigenvectors into real and imaginary parts (a conjugate pair then contributes two
    columns, so k may grow by one), orthonormalise -> P_k (mp x k').

    ``align`` (a reading for a block method: the paper lets k "be increased or decreased"):
    the kept count is a multiple of align.  k is rounded up to a multiple of align; Ritz
    values are walked in wanted order with a conjugate pair as one group of two columns; a
    group is kept only if it still fits, so a pair that does not fit is skipped in favour of
    the next real value; if the count is then not a multiple of align, the least wanted
    groups are dropped until it is."""
    theta, Y = np.linalg.eig(Hm)
    order = list(np.argsort(-np.abs(theta), kind="stable") if largest else
                 np.argsort(np.abs(theta), kind="stable"))
    # groups in wanted order: a real value, or a conjugate pair (its Im > 0 member's vector)
    groups, taken = [], set()
    for idx in order:
        if idx in taken:
            continue
        taken.add(idx)
        if abs(theta[idx].imag) > 1e-12 * max(abs(theta[idx]), 1e-300):
            rest = [j for j in order if j not in taken]
            partner = min(rest, key=lambda j: abs(theta[j] - np.conj(theta[idx])))
            taken.add(partner)
            y = Y[:, idx] if theta[idx].imag > 0 else Y[:, partner]
            groups.append([y.real, y.imag])
        else:
            groups.append([Y[:, idx].real])
    if align is None:
        cols = []
        for gcols in groups:
            if len(cols) >= k:
                break
            cols += gcols
    else:
        target = min(Hm.shape[0], -(-k // align) * align)
        sel, count = [], 0
        for gcols in groups:
            if count + len(gcols) <= target:
                sel.append(gcols)
                count += len(gcols)
            if count == target:
                break
        while count % align != 0 and sel:
            count -= len(sel.pop())
        cols = [c for gcols in sel for c in gcols]
        if not cols:
            return np.zeros((Hm.shape[0], 0))
    Q, _ = np.linalg.qr(np.column_stack(cols))
    return Q


# --------------------------------------------------------------------------- Algorithm 2
def psbfom(apply_Ainv, B, table, m=10, tol=1e-10, max_cycles=100, k=0, fixed_cycles=None,
           return_details=False, align=None):
    """Algorithm 2 (PSBFOM[-DR]) for Z ~= e^A B, A already scaled by t.

    apply_Ainv : callable, w (n,) -> A^{-1} w  (the right preconditioner M_i = A^{-1})
    B          : (n, p) real
    table      : CF table with 'tau' (Im > 0 poles), 'omega', 'omega0'
    k          : number of deflated Ritz vectors (0 = plain restart)
    align      : keep a multiple of this many Ritz vectors (see deflation_basis)
    fixed_cycles : run exactly this many cycles (ignores tol), for parity tests
    """
    B = np.asarray(B, dtype=np.float64)
    n, p = B.shape
    taus = np.asarray(table["tau"])
    omegas = np.asarray(table["omega"])
    nup = len(taus)
    normB = np.linalg.norm(B)
    # initial guesses Y_i^0 = O
    Y = [np.zeros((n, p), dtype=complex) for _ in range(nup)]
    # QR of the common initial residual R_i^0 = B
    V1, R = qr_positive(B)
    Rhat = [R.astype(complex) for _ in range(nup)]
    history = []
    cycles = 0
    matvecs = 0
    start_vectors = None
    H0 = None
    rhs_row0 = 0            # block row of the residual coordinates (0, or k/p after deflation)
    converged = False
    details = []
    while True:
        cycles += 1
        # block Arnoldi with the Krylov operator A^{-1}  (eq. (4.5))
        V, Ht, m_done, breakdown = block_arnoldi_ruhe(apply_Ainv, V1, m, start_vectors, H0)
        first = p if start_vectors is None else start_vectors.shape[1]
        matvecs += (m_done + 1) * p - first
        mp_ = m_done * p
        Hm = Ht[:mp_, :mp_]
        Hlast = Ht[mp_:mp_ + p, mp_ - p:mp_]           # H_{m+1,m}
        Vm = V[:, :mp_]
        # projected systems (I - tau_i H_m) Z_i = E_1 R_i  (eq. (3236))
        res = np.zeros(nup)
        Zhat = []
        for i in range(nup):
            rhs = np.zeros((mp_, p), dtype=complex)
            rhs[rhs_row0:rhs_row0 + p, :] = Rhat[i]
            Zi = np.linalg.solve(np.eye(mp_) - taus[i] * Hm, rhs)
            Zhat.append(Zi)
            Y[i] = Y[i] + Vm @ Zi
            # eq. (49): ||R_i||_F = |tau_i| ||H_{m+1,m} E_m^T Z_i||_F
            res[i] = abs(taus[i]) * np.linalg.norm(Hlast @ Zi[mp_ - p:, :])
        history.append(res.copy())
        if return_details:
            details.append({"V": V, "H": Ht, "Zhat": Zhat, "res": res.copy()})
        if fixed_cycles is not None:
            done = cycles >= fixed_cycles
        else:
            done = res.max() <= tol * normB or cycles >= max_cycles or breakdown
        converged = res.max() <= tol * normB
        if done or breakdown:
            break
        # restart: residuals tau_i V_{m+1} H_{m+1,m} E_m^T Z_i are collinear with V_{m+1}
        Vnext = V[:, mp_:mp_ + p]
        Snew = [taus[i] * (Hlast @ Zhat[i][mp_ - p:, :]) for i in range(nup)]
        Pk = deflation_basis(Hm, k, largest=True, align=align) if k > 0 else None
        if Pk is not None and Pk.shape[1] > 0:
            # the deflated restart of Algorithm 1, with A^{-1} as the operator
            kk = Pk.shape[1]
            Pk1 = np.zeros(((m_done + 1) * p, kk + p))
            Pk1[:mp_, :kk] = Pk
            Pk1[mp_:, kk:] = np.eye(p)
            Hnew = Pk1.T @ Ht @ Pk                     # (k+p) x k
            Vnew = V @ Pk1                              # n x (k+p)
            start_vectors = Vnew
            H0 = Hnew
            # residual coordinates: R_i = V_{m+1} S_i = Vnew[:, k:k+p] S_i (reading:
            # the right-hand side of eq. (3236) sits in rows k..k+p-1 after deflation)
            rhs_row0 = kk
            V1 = Vnew[:, kk:kk + p]
            Rhat = Snew
        else:
            V1 = Vnext
            Rhat = Snew
            rhs_row0 = 0
    # form the numerical solutions X_i = A^{-1} Y_i and Z = omega_0 B + sum 2 Re(omega_i X_i)
    Z = table["omega0"] * B
    X = []
    for i in range(nup):
        Xi_re = np.column_stack([apply_Ainv(Y[i][:, c].real) for c in range(p)])
        Xi_im = np.column_stack([apply_Ainv(Y[i][:, c].imag) for c in range(p)])
        Xi = Xi_re + 1j * Xi_im
        X.append(Xi)
        Z = Z + 2.0 * np.real(omegas[i] * Xi)
    info = {"cycles": cycles, "block_steps": matvecs / p, "matvecs": matvecs,
            "residuals": history, "converged": converged, "breakdown": breakdown,
            "X": X}
    if return_details:
        info["details"] = details
    return Z, info


# --------------------------------------------------------------------------- Algorithm 1
def sbfom(apply_A, B, table, m=10, tol=1e-10, max_cycles=1000, fixed_cycles=None, k=0, align=None):
    """Algorithm 1 (SBFOM[-DR]): the unpreconditioned shifted block FOM.

    k     : number of deflated Ritz vectors (0 = plain restart): the k smallest |theta| of H_m
    align : keep a multiple of this many Ritz vectors (see deflation_basis)"""
    B = np.asarray(B, dtype=np.float64)
    n, p = B.shape
    taus = np.asarray(table["tau"])
    omegas = np.asarray(table["omega"])
    nup = len(taus)
    normB = np.linalg.norm(B)
    X = [np.zeros((n, p), dtype=complex) for _ in range(nup)]
    V1, R = qr_positive(B)
    Rhat = [R.astype(complex) for _ in range(nup)]
    history = []
    cycles = 0
    matvecs = 0
    converged = False
    start_vectors = None
    H0 = None
    rhs_row0 = 0
    while True:
        cycles += 1
        V, Ht, m_done, breakdown = block_arnoldi_ruhe(apply_A, V1, m, start_vectors, H0)
        first = p if start_vectors is None else start_vectors.shape[1]
        matvecs += (m_done + 1) * p - first
        mp_ = m_done * p
        Hm = Ht[:mp_, :mp_]
        Hlast = Ht[mp_:mp_ + p, mp_ - p:mp_]
        res = np.zeros(nup)
        Snew = []
        for i in range(nup):
            rhs = np.zeros((mp_, p), dtype=complex)
            rhs[rhs_row0:rhs_row0 + p, :] = Rhat[i]
            Zi = np.linalg.solve(Hm - taus[i] * np.eye(mp_), rhs)      # eq. (3.3)
            X[i] = X[i] + V[:, :mp_] @ Zi
            S = -(Hlast @ Zi[mp_ - p:, :])                             # eq. (35)
            res[i] = np.linalg.norm(S)                                  # eq. (365)
            Snew.append(S)
        history.append(res.copy())
        converged = res.max() <= tol * normB
        if fixed_cycles is not None:
            if cycles >= fixed_cycles:
                break
        elif converged or cycles >= max_cycles or breakdown:
            break
        Pk = deflation_basis(Hm, k, largest=False, align=align) if k > 0 else None
        if Pk is not None and Pk.shape[1] > 0:
            # the deflated restart: V_new = V_{m+1} blkdiag(P_k, I_p), H_new = its projection;
            # the residuals stay collinear with V_{m+1}, now the columns kk..kk+p-1
            kk = Pk.shape[1]
            Pk1 = np.zeros(((m_done + 1) * p, kk + p))
            Pk1[:mp_, :kk] = Pk
            Pk1[mp_:, kk:] = np.eye(p)
            H0 = Pk1.T @ Ht @ Pk
            start_vectors = V @ Pk1
            rhs_row0 = kk
            V1 = start_vectors[:, kk:kk + p]
        else:
            V1 = V[:, mp_:mp_ + p]
            start_vectors, H0, rhs_row0 = None, None, 0
        Rhat = Snew
    Z = table["omega0"] * B
    for i in range(nup):
        Z = Z + 2.0 * np.real(omegas[i] * X[i])
    return Z, {"cycles": cycles, "block_steps": matvecs / p, "matvecs": matvecs,
               "residuals": history, "converged": converged, "X": X}


# --------------------------------------------------------------------------- truths
def dense_r_of_A_B(A, B, table):
    """r(A) B = omega_0 B + sum_i 2 Re(omega_i (A - tau_i I)^{-1} B) by dense solves
    (eq. (11)); only for small n."""
    A = np.asarray(A.todense() if hasattr(A, "todense") else A, dtype=np.float64)
    n = A.shape[0]
    Z = table["omega0"] * B
    for tau, om in zip(table["tau"], table["omega"]):
        Xi = np.linalg.solve(A - tau * np.eye(n), B.astype(complex))
        Z = Z + 2.0 * np.real(om * Xi)
    return Z
