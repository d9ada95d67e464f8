"""The launch-latency plus bandwidth model of Sec. 4 and its least-squares fit.

T(B) = T0 + B / Wmax                          (eq. time_model)
W_eff(B) = B / (T0 + B / Wmax)                (eq. perf_model)
B_0.8 = 4 T0 Wmax, where W_eff = 0.8 Wmax    (eq. Fischer-Brown)

The fit is the paper's: an ordinary least-squares line through the measured
(bytes, seconds) pairs of every trial (Sec. 6.2), intercept T0, slope 1/Wmax.
"""
from __future__ import annotations

import numpy as np


def time_model(B, T0: float, Wmax: float):
    """Seconds to stream B bytes (eq. time_model)."""
    return T0 + np.asarray(B, dtype=np.float64) / Wmax


def effective_bandwidth(B, T0: float, Wmax: float):
    """Bytes per second achieved when streaming B bytes (eq. perf_model)."""
    B = np.asarray(B, dtype=np.float64)
    return B / (T0 + B / Wmax)


def fischer_brown(T0: float, Wmax: float, fraction: float = 0.8) -> float:
    """Bytes needed to reach `fraction` of Wmax: f T0 Wmax / (1 - f);
    for f = 0.8 this is 4 T0 Wmax (eq. Fischer-Brown)."""
    return fraction * T0 * Wmax / (1.0 - fraction)


def fit(bytes_moved, seconds):
    """Least-squares fit of eq. time_model: returns (T0 seconds, Wmax B/s)."""
    B = np.asarray(bytes_moved, dtype=np.float64)
    T = np.asarray(seconds, dtype=np.float64)
    A = np.stack([np.ones_like(B), B], axis=1)
    (t0, inv_w), *_ = np.linalg.lstsq(A, T, rcond=None)
    return float(t0), float(1.0 / inv_w)
