"""Pins for the oracle's Magnus predictor-corrector propagation (Eqs. 25-26, Sec. VI.B)."""
import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle.ground_state import lowest_states, scf
from oracle.mesh import Mesh
from oracle.propagate import Propagator, kick, nuclear_potential


def _box(L, n, p):
    b = np.linspace(-L, L, n + 1)
    return Mesh(b, b, b, p)


def test_kicked_harmonic_oscillator_closed_form():
    """Non-interacting V = w^2 r^2 / 2, ground state kicked by exp(-i k z):
    <z>(t) = -(k / w) sin(w t) per electron (exact: the Magnus step is exact for a
    time-independent Hamiltonian, so only the FE and Krylov errors remain)."""
    m = _box(7.0, 4, 6)
    w, kap = 1.0, 0.1
    vn = nuclear_potential(m, "harmonic", [[0, 0, 0]], [0], w)
    _, psi = lowest_states(m, vn, 1)
    prop = Propagator(m, vn, [2.0], hartree=False, use_xc=False)
    ps = kick(m, psi.astype(complex), kap, (0, 0, 1))
    prop.init(ps)
    T = 0.0
    for _ in range(4):
        ps, d, _ = prop.magnus_step(ps, 0.25)
        T += 0.25
        ex = -2.0 * kap / w * np.sin(w * T)
        assert abs(d[2] - ex) < 5e-4 * abs(ex)
        assert abs(d[0]) < 1e-12 and abs(d[1]) < 1e-12


def test_harmonic_potential_theorem_interacting():
    """With Hartree + ALDA the kicked dipole of a harmonic well still follows
    -N_e (k / w) sin(w t) (harmonic potential theorem); the grounded box and the
    FE mesh break it only slightly."""
    m = _box(7.0, 3, 6)
    w, kap = 1.0, 0.05
    vn = nuclear_potential(m, "harmonic", [[0, 0, 0]], [0], w)
    psi, _, _ = scf(m, vn, [2.0], 1, n_iter=15)
    prop = Propagator(m, vn, [2.0])
    ps = kick(m, psi.astype(complex), kap, (0, 0, 1))
    prop.init(ps)
    T = 0.0
    for _ in range(10):
        ps, d, _ = prop.magnus_step(ps, 0.1)
        T += 0.1
        ex = -2.0 * kap / w * np.sin(w * T)
        assert abs(d[2] - ex) < 0.015 * (2.0 * kap / w)


def test_dipole_converges_at_second_order_in_dt():
    """Eq. 29: the full-discrete error is O(Dt^2); the paper measures q = 1.96-1.98."""
    m = _box(6.0, 3, 4)
    vn = nuclear_potential(m, "soft", [[0, 0, 0]], [2.0], 0.5)
    psi, _, _ = scf(m, vn, [2.0], 1, n_iter=10)
    E = lambda t: np.array([0.0, 0.0, 0.05 * np.sin(1.3 * t)])
    res = {}
    for dt in (0.2, 0.1, 0.05, 0.0125):
        prop = Propagator(m, vn, [2.0])
        ps = psi.astype(complex).copy()
        prop.init(ps)
        for s in range(int(round(1.0 / dt))):
            t0 = s * dt
            ps, d, _ = prop.magnus_step(ps, dt, E(t0 + dt / 4), E(t0 + dt / 2))
        res[dt] = d[2]
    errs = [abs(res[dt] - res[0.0125]) for dt in (0.2, 0.1, 0.05)]
    q1, q2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.8 < q1 < 2.3 and 1.8 < q2 < 2.4


def test_unitarity_and_orthonormality():
    m = _box(5.0, 2, 4)
    vn = nuclear_potential(m, "soft", [[0.2, 0, 0], [-0.3, 0.1, 0]], [2.0, 2.0], 0.5)
    _, psi = lowest_states(m, vn, 2)
    prop = Propagator(m, vn, [2.0, 2.0])
    ps = kick(m, psi.astype(complex), 1e-2, (1, 0, 0))
    prop.init(ps)
    n0 = 4.0
    for _ in range(5):
        ps, _, _ = prop.magnus_step(ps, 0.1)
    G = ps.conj() @ ps.T
    assert np.abs(G - np.eye(2)).max() < 1e-9
    assert abs(np.sum(prop.occ * np.sum(np.abs(ps) ** 2, axis=1)) - n0) < 1e-9
