"""Absorption spectrum from a kicked dipole series (oracle).

Test infrastructure only (see oracle/__init__.py).

Sec. VII (Al2 example): the dynamic polarizability alpha_ab(omega) is the Fourier
transform of the dipole response, broadened by a Gaussian window g(t) = exp(-alpha t^2),
and the dipole strength function is S(omega) = (2 omega / 3 pi) Tr Im alpha(omega).

Kick convention (reading of Sec. VII.A): psi(0) = exp(-i kappa r.d) psi_GS is the impulse
of a field E(t) = -kappa d delta(t) (V_field = -E.r), so the linear response is
d_b(t) - d_b(0) = -kappa alpha_{ab}(t) and
    alpha_ab(omega) = -(1 / kappa) int_0^T exp(i omega t) g(t) (d_b(t) - d_b(0)) dt,
the time integral by the trapezoid rule on the sampled steps t_n = n dt.
"""
from __future__ import annotations

import numpy as np


def polarizability(dip, dt: float, kappa: float, direction, omega) -> np.ndarray:
    """alpha_aa(omega) for the kick direction a (dip: [n_steps+1, 3], d(t_n))."""
    dip = np.asarray(dip, float)
    a = np.asarray(direction, float)
    a = a / np.linalg.norm(a)
    resp = dip @ a - dip[0] @ a                       # d_a(t_n) - d_a(0)
    t = dt * np.arange(len(resp))
    w = np.full(len(resp), dt)
    w[0] = w[-1] = 0.5 * dt                            # trapezoid weights
    omega = np.atleast_1d(np.asarray(omega, float))
    return np.array([-(1.0 / kappa) * np.sum(w * np.exp(1j * om * t) * resp) for om in omega])


def windowed(dip, window_alpha: float, dt: float) -> np.ndarray:
    """The dipole series with d(t) - d(0) multiplied by g(t) = exp(-alpha t^2)."""
    dip = np.asarray(dip, float)
    t = dt * np.arange(len(dip))
    g = np.exp(-window_alpha * t * t)
    return dip[0][None, :] + (dip - dip[0][None, :]) * g[:, None]


def strength(series, dt: float, kappa: float, window_alpha: float, omega) -> np.ndarray:
    """S(omega) = (2 omega / 3 pi) sum_a Im alpha_aa(omega) over the kicked series given
    as [(dipoles, direction), ...] (one per kick direction; three for the full trace)."""
    omega = np.atleast_1d(np.asarray(omega, float))
    tr = np.zeros(len(omega))
    for dip, direction in series:
        tr += polarizability(windowed(dip, window_alpha, dt), dt, kappa, direction, omega).imag
    return 2.0 * omega / (3.0 * np.pi) * tr
