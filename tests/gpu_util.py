"""Helpers for the GPU parity tests (imported by tests only)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_0707_gb300 import _native as N
    N.load(build_if_missing=True)
    return torch


def to_dev(X):
    from paper_1405_0707_gb300.inputs import to_device_colmajor
    return to_device_colmajor(np.asarray(X, dtype=np.float64))


def to_np(X):
    return X.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cancellation_floor(tab, X, Z):
    """eps * sum_i 2|omega_i| ||X_i|| / ||Z||: two FP64 evaluations of the partial-fraction
    sum (eq. (11)) can differ by this much however accurate each X_i is."""
    s = sum(2 * abs(o) * np.linalg.norm(x) for o, x in zip(tab["omega"], X))
    return np.finfo(float).eps * s / np.linalg.norm(Z)


def closed_form_poles(sides, diff, vel, t, tab, B):
    """X_i = (tA - tau_i I)^{-1} B for every pole with Im tau > 0, by the oracle's closed-form
    eigen-expansion (diagonal similarity + DST-I; no Krylov iteration involved)."""
    from oracle import operators as ops
    return [ops.apply_function(sides, diff, vel, t, lambda lam, z=z: 1.0 / (lam - z), B)
            for z in tab["tau"]]


def closed_form_floor(sides, diff, vel, t, tab, B, Z):
    """cancellation_floor with the X_i taken from the closed form (cheap at any size)."""
    return cancellation_floor(tab, closed_form_poles(sides, diff, vel, t, tab, B), Z)
