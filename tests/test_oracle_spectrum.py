"""Pins for the absorption-spectrum post-processing: the windowed Fourier transform of a
single damped mode against its closed form, linearity, and the trace over three kicks."""
import numpy as np

from oracle import spectrum


def _mode(kappa, w0, amp, dt, n):
    """Dipole of a single mode after a kick along z: d_z(t) = d0 - kappa amp sin(w0 t)."""
    t = dt * np.arange(n + 1)
    d = np.zeros((n + 1, 3))
    d[:, 2] = 0.7 - kappa * amp * np.sin(w0 * t)
    return d


def test_single_mode_closed_form():
    # Im int_0^inf e^{i w t} e^{-a t^2} A sin(w0 t) dt
    #   = (A / 4) sqrt(pi / a) (exp(-(w - w0)^2 / 4a) - exp(-(w + w0)^2 / 4a))
    kappa, w0, amp, a, dt = 1e-3, 0.45, 2.0, 0.005, 0.01
    n = 6000                                  # T = 60: e^{-a T^2} = 1.5e-8
    d = _mode(kappa, w0, amp, dt, n)
    om = np.linspace(0.2, 0.7, 11)
    alpha = spectrum.polarizability(spectrum.windowed(d, a, dt), dt, kappa, (0, 0, 1), om)
    ref = amp / 4 * np.sqrt(np.pi / a) * (np.exp(-(om - w0) ** 2 / (4 * a)) - np.exp(-(om + w0) ** 2 / (4 * a)))
    np.testing.assert_allclose(alpha.imag, ref, atol=2e-6 * np.abs(ref).max())
    S = spectrum.strength([(d, (0, 0, 1))], dt, kappa, a, om)
    np.testing.assert_allclose(S, 2 * om / (3 * np.pi) * ref, atol=2e-6 * np.abs(ref).max())


def test_linear_in_the_response_and_independent_of_the_static_dipole():
    kappa, dt, n = 1e-3, 0.05, 400
    d1 = _mode(kappa, 0.3, 1.0, dt, n)
    d2 = _mode(kappa, 0.8, 0.5, dt, n)
    dsum = d1 + d2
    om = np.array([0.1, 0.3, 0.5, 0.8])
    a1 = spectrum.polarizability(d1, dt, kappa, (0, 0, 1), om)
    a2 = spectrum.polarizability(d2, dt, kappa, (0, 0, 1), om)
    a12 = spectrum.polarizability(dsum, dt, kappa, (0, 0, 1), om)
    np.testing.assert_allclose(a12, a1 + a2, rtol=1e-12, atol=1e-12)
    shifted = d1 + np.array([3.0, -1.0, 5.0])[None, :]
    np.testing.assert_allclose(spectrum.polarizability(shifted, dt, kappa, (0, 0, 1), om), a1,
                               rtol=1e-12, atol=1e-12)


def test_trace_over_three_kicks():
    kappa, dt, n, a = 1e-3, 0.02, 2000, 0.01
    om = np.linspace(0.1, 1.0, 7)
    series = []
    for k, w0 in enumerate((0.3, 0.5, 0.7)):
        t = dt * np.arange(n + 1)
        d = np.zeros((n + 1, 3))
        d[:, k] = -kappa * np.sin(w0 * t)
        e = np.zeros(3)
        e[k] = 1.0
        series.append((d, e))
    S = spectrum.strength(series, dt, kappa, a, om)
    parts = sum(spectrum.strength([s], dt, kappa, a, om) for s in series)
    np.testing.assert_allclose(S, parts, rtol=1e-12)
    assert np.all(S > -1e-12)                 # a positive mode gives a positive strength
