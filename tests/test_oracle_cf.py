"""Pins for the oracle's Caratheodory-Fejer table (paper Section 2, Remark 2.1).

The stored table tests/golden/cf_nu14.json is written by oracle/make_cf_table.py.  It is
pinned against facts outside the oracle's own code:
  * Remark 2.1: for nu = 14, max_i |tau_i| is about 18.9;
  * the mathematics of the approximation: r(x) must match e^x on (-inf, 0] to the CF
    error sigma (the (nu+1)-st Hankel singular value), and a near-best type (nu, nu)
    approximant's error curve alternates in sign 2 nu + 2 = 30 times with nearly equal
    extrema (Chebyshev equioscillation; the CF approximant differs from the best one by
    O(56^-nu), Section 2).  A dropped pole, a wrong sign or a swapped real/imaginary part
    of a residue destroys both properties.
"""
import numpy as np
import pytest

from oracle import cf


def _err_curve(tab, npts=400001):
    w = np.linspace(-1, 1, npts, dtype=np.longdouble)[1:]
    x = 9 * (w - 1) / (w + 1)
    r = np.full(x.shape, np.longdouble(tab["omega0"]))
    for t, o in zip(tab["tau"], tab["omega"]):
        dr = x - np.longdouble(t.real)
        ti = np.longdouble(t.imag)
        r += 2 * (np.longdouble(o.real) * dr - np.longdouble(o.imag) * ti) / (dr * dr + ti * ti)
    return x, (r - np.exp(x)).astype(np.float64)


def _alternations(e, level):
    sg = np.sign(e[np.abs(e) > level])
    return 1 + int(np.count_nonzero(sg[1:] != sg[:-1]))


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def test_remark_2_1_max_pole_modulus(tab):
    # Remark 2.1: "max |tau_i| ~ 18.9" for nu = 14
    assert len(tab["tau"]) == 7 and np.all(tab["tau"].imag > 0)
    assert abs(np.abs(tab["tau"]).max() - 18.9) < 0.05


def test_error_matches_cf_singular_value(tab):
    _, e = _err_curve(tab)
    emax = np.abs(e).max()
    assert 1.0e-14 < tab["sigma"] < 3.0e-14
    assert emax < 1.1 * tab["sigma"]          # near-best: within 10 % of sigma
    assert abs(tab["omega0"]) < 1.1 * tab["sigma"]   # r(-inf) = omega_0 ~ 0 = e^-inf


def test_equioscillation(tab):
    _, e = _err_curve(tab)
    s = tab["sigma"]
    assert _alternations(e, 0.5 * s) == 2 * 7 * 2 + 2     # 2 nu + 2 = 30
    # each alternation's extremum is within 10 % of sigma
    mask = np.abs(e) > 0.5 * s
    ev = e[mask]
    cuts = np.flatnonzero(np.sign(ev[1:]) != np.sign(ev[:-1])) + 1
    ext = [np.abs(seg).max() for seg in np.split(ev, cuts)]
    assert min(ext) > 0.9 * s and max(ext) < 1.1 * s


def test_r_at_zero_and_far_left(tab):
    x, e = _err_curve(tab, 20001)
    assert abs(e[-1]) < 1.1 * tab["sigma"]            # x = 0: r(0) ~ 1
    xs = np.array([-1e3, -1e6, -1e9])
    from oracle.operators import r_of_lambda_ext
    assert np.all(np.abs(r_of_lambda_ext(tab, xs)) < 2 * tab["sigma"])


@pytest.mark.slow
def test_recompute_matches_stored_and_is_scale_free(tab):
    """Recompute at a different transplant scale s and smaller K: the poles do not depend
    on s (checked for s = 6..12) and the Hankel truncation at K = 80 is already converged
    to well below FP64 resolution."""
    pytest.importorskip("mpmath")
    import mpmath as mp
    with mp.workdps(40):
        upper, sigma = cf.cf_poles(nu=14, s=7, K=80, N=512)
    tau7 = np.array([complex(t) for t in upper])
    assert np.max(np.abs(tau7 - tab["tau"]) / np.abs(tab["tau"])) < 1e-13
    assert abs(float(sigma) - tab["sigma"]) < 1e-6 * tab["sigma"]


def test_planted_mistakes_fail_the_pins(tab):
    """A plausible mistake in the table (dropped pole, sign flip, conjugated residue)
    must break the approximation pin."""
    bad = []
    t1 = dict(tab); t1["tau"] = tab["tau"][1:]; t1["omega"] = tab["omega"][1:]; bad.append(t1)
    t2 = dict(tab); t2["omega"] = tab["omega"].copy(); t2["omega"][3] *= -1; bad.append(t2)
    t3 = dict(tab); t3["omega"] = np.conj(tab["omega"]); bad.append(t3)
    t4 = dict(tab); t4["tau"] = np.conj(tab["tau"]); bad.append(t4)
    for b in bad:
        _, e = _err_curve(b, 20001)
        assert np.abs(e).max() > 100 * tab["sigma"]


def _err_curve_strings(tab, npts=400001):
    """The error curve with the coefficients taken from their stored 25-digit strings in
    extended precision (for nu = 16 the FP64 rounding of the residues alone is ~1e-14, far
    above its sigma ~ 3e-16)."""
    L = np.longdouble
    w = np.linspace(-1, 1, npts, dtype=L)[1:]
    x = 9 * (w - 1) / (w + 1)
    r = np.full(x.shape, L(tab["omega0_str"]))
    for (tr, ti), (orr, oi) in zip(tab["tau_str"], tab["omega_str"]):
        dr = x - L(tr)
        tiL = L(ti)
        r += 2 * (L(orr) * dr - L(oi) * tiL) / (dr * dr + tiL * tiL)
    return x, (r - np.exp(x)).astype(np.float64)


@pytest.mark.parametrize("nu", [10, 12, 16])
def test_other_degrees_are_near_best(nu):
    """The stored tables of the degrees a plan may choose (nu_cf): error at most 1.1 sigma on
    (-inf, 0], 2 nu + 2 alternations with extrema within 10 % of sigma, nu/2 poles in the upper
    half-plane."""
    tab = cf.load_table(nu=nu)
    assert tab["nu"] == nu and len(tab["tau"]) == nu // 2 and np.all(tab["tau"].imag > 0)
    _, e = _err_curve_strings(tab)
    s = tab["sigma"]
    assert np.abs(e).max() < 1.1 * s, (nu, np.abs(e).max(), s)
    assert _alternations(e, 0.5 * s) == 2 * nu + 2
    mask = np.abs(e) > 0.5 * s
    ev = e[mask]
    cuts = np.flatnonzero(np.sign(ev[1:]) != np.sign(ev[:-1])) + 1
    ext = [np.abs(seg).max() for seg in np.split(ev, cuts)]
    assert min(ext) > 0.9 * s and max(ext) < 1.1 * s
