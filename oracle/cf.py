"""Caratheodory-Fejer (CF) rational approximation of e^x on (-inf, 0]  -- ORACLE.

Test infrastructure only (see ``oracle/__init__.py``).  High-precision (mpmath) and
slow on purpose; the product library computes the same table with its own code.

Paper, Section 2: the CF approximant is built from the singular value decomposition of
a Hankel matrix of the Chebyshev coefficients of e^x transplanted from R^- to [-1, 1];
the result is written in partial-fraction form

    r(x) = omega_0 + sum_{i=1..nu} omega_i / (x - tau_i)                    (Section 2)

and e^A B is replaced by  omega_0 B + sum_i omega_i (A - tau_i I)^{-1} B  (eq. (11)).
For real data the poles come in conjugate pairs, so only the nu/2 poles in the upper
half-plane are kept and  r(x) = omega_0 + sum_{Im tau>0} 2 Re(omega_i / (x - tau_i)).

The paper gives no algorithmic detail beyond that sentence, so the steps below are the
textbook Chebyshev-CF construction, each step written out:

 1. transplant:  x = s (w - 1) / (w + 1)  maps w in [-1, 1] onto x in [-inf, 0];
    F(w) = exp(x(w)).  The scale s is a free parameter (the poles were checked to be
    independent of s for s in 6..12 to >= 12 digits); s = 9.
 2. Chebyshev coefficients c_k of F, k = 0..K, by the trapezoidal rule on the
    N + 1 Chebyshev-Lobatto points w_j = cos(pi j / N).
 3. the K x K Hankel matrix  H[i, j] = c_{i+j+1}  (zero when i + j + 1 > K); it is
    real symmetric, so its singular values are the |eigenvalues|.  Take the
    eigenpair with the (nu+1)-st largest |lambda|:  sigma = |lambda|, vector v.
 4. the CF denominator is the polynomial  q(z) = sum_j v_j z^(K-1-j); exactly nu of
    its roots lie outside the unit disk.  A root z maps to w = (z + 1/z)/2 and then
    to the pole  tau = s (z - 1)^2 / (z + 1)^2  in the x-plane.
 5. residues (a reading: the paper does not say how): with the poles fixed, omega_0 and the
    omega_i are the linear least-squares fit of e^x on the M Chebyshev points of the
    first kind in w, plus the point w = -1 (x = -inf) where e^x = 0.
"""
from __future__ import annotations

import json
import os

import numpy as np

try:  # mpmath is needed only to (re)compute the table, not to use a stored one
    import mpmath as mp
except ImportError:  # pragma: no cover - the GPU machine may lack it
    mp = None

NU_DEFAULT = 14
S_DEFAULT = 9
K_DEFAULT = 100
N_DEFAULT = 1024
M_DEFAULT = 512
GOLDEN_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
GOLDEN = os.path.join(GOLDEN_DIR, "cf_nu14.json")


def golden_path(nu):
    """Stored table of degree nu (written by oracle/make_cf_table.py)."""
    return os.path.join(GOLDEN_DIR, "cf_nu%d.json" % nu)


def _transplant(s, w):
    """Step 1: x(w) = s (w - 1)/(w + 1); e^x is 0 at w = -1 (x = -inf)."""
    if w == -1:
        return None
    return s * (w - 1) / (w + 1)


def chebyshev_coefficients(s, K, N):
    """Step 2: c_k, k = 0..K, of F(w) = exp(s (w-1)/(w+1)) on [-1, 1].

    c_k = (2/N) sum''_{j=0..N} F(cos(pi j/N)) cos(pi j k/N), with c_0 halved;
    '' halves the two end terms (trapezoidal rule in theta = arccos w).
    """
    theta = [mp.pi * j / N for j in range(N + 1)]
    F = []
    for th in theta:
        x = _transplant(s, mp.cos(th))
        F.append(mp.mpf(0) if x is None else mp.exp(x))
    c = []
    for k in range(K + 1):
        acc = mp.mpf(0)
        for j in range(N + 1):
            term = F[j] * mp.cos(k * theta[j])
            acc += term / 2 if j in (0, N) else term
        c.append(2 * acc / N)
    c[0] /= 2
    return c


def cf_poles(nu=NU_DEFAULT, s=S_DEFAULT, K=K_DEFAULT, N=N_DEFAULT):
    """Steps 2-4.  Returns (upper-half-plane poles sorted by decreasing Im, sigma)."""
    s = mp.mpf(s)
    c = chebyshev_coefficients(s, K, N)
    H = mp.matrix(K, K)
    for i in range(K):
        for j in range(K):
            if i + j + 1 <= K:
                H[i, j] = c[i + j + 1]
    evals, evecs = mp.eigsy(H)
    order = sorted(range(K), key=lambda i: -abs(evals[i]))
    sigma = abs(evals[order[nu]])
    v = [evecs[j, order[nu]] for j in range(K)]
    roots = mp.polyroots(v, maxsteps=800, extraprec=300)
    outside = [z for z in roots if abs(z) > 1]
    if len(outside) != nu:
        raise RuntimeError(f"expected {nu} roots outside the unit disk, got {len(outside)}")
    poles = [s * (z - 1) ** 2 / (z + 1) ** 2 for z in outside]
    upper = sorted([t for t in poles if mp.im(t) > 0], key=lambda t: -mp.im(t))
    if len(upper) != nu // 2:
        raise RuntimeError("poles are not in conjugate pairs")
    return upper, sigma


def ls_residues(upper, s=S_DEFAULT, M=M_DEFAULT):
    """Step 5: real least squares for (omega_0, Re omega_i, Im omega_i).

    Model on real x:  omega_0 + sum_i 2 [Re(omega_i) Re(1/(x - tau_i))
                                         - Im(omega_i) Im(1/(x - tau_i))].
    Rows: w_j = cos(pi (j + 1/2) / M), j = 0..M-1, target e^{x(w_j)}; one extra row
    at x = -inf where the model is omega_0 and the target is 0.
    """
    s = mp.mpf(s)
    rows, rhs = [], []
    for j in range(M):
        w = mp.cos(mp.pi * (j + mp.mpf(1) / 2) / M)
        x = _transplant(s, w)
        row = [mp.mpf(1)]
        for t in upper:
            g = 1 / (x - t)
            row += [2 * mp.re(g), -2 * mp.im(g)]
        rows.append(row)
        rhs.append(mp.exp(x))
    rows.append([mp.mpf(1)] + [mp.mpf(0)] * (2 * len(upper)))
    rhs.append(mp.mpf(0))
    sol = mp.qr_solve(mp.matrix(rows), mp.matrix(rhs))[0]
    omega0 = sol[0]
    omega = [sol[1 + 2 * i] + 1j * sol[2 + 2 * i] for i in range(len(upper))]
    return omega0, omega


def cf_table(nu=NU_DEFAULT, s=S_DEFAULT, K=K_DEFAULT, N=N_DEFAULT, M=M_DEFAULT, dps=50):
    """Full table (steps 1-5) at ``dps`` decimal digits; values returned as Python
    complex/float rounded to FP64 plus 25-digit strings."""
    if mp is None:
        raise RuntimeError("mpmath is required to compute the CF table")
    with mp.workdps(dps):
        upper, sigma = cf_poles(nu, s, K, N)
        omega0, omega = ls_residues(upper, s, M)
        return {
            "nu": nu, "s": s, "K": K, "N": N, "M": M,
            "tau": [complex(t) for t in upper],
            "omega": [complex(w) for w in omega],
            "omega0": float(omega0),
            "sigma": float(sigma),
            "tau_str": [(mp.nstr(mp.re(t), 25), mp.nstr(mp.im(t), 25)) for t in upper],
            "omega_str": [(mp.nstr(mp.re(w), 25), mp.nstr(mp.im(w), 25)) for w in omega],
            "omega0_str": mp.nstr(omega0, 25),
        }


def load_table(path=GOLDEN, nu=None):
    """Stored table written by ``oracle/make_cf_table.py`` (which calls only this module);
    ``nu`` picks the stored table of that degree instead of ``path``."""
    if nu is not None:
        path = golden_path(nu)
    with open(path) as f:
        d = json.load(f)
    return {
        "nu": d["nu"],
        "tau": np.array([complex(float(a), float(b)) for a, b in d["tau_str"]]),
        "omega": np.array([complex(float(a), float(b)) for a, b in d["omega_str"]]),
        "omega0": float(d["omega0_str"]),
        "sigma": float(d["sigma"]),
        "tau_str": d["tau_str"], "omega_str": d["omega_str"], "omega0_str": d["omega0_str"],
    }
