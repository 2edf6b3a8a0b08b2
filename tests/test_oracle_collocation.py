"""Pins for the GLL-collocation variant of Hbar: GLL quadrature is exact for the kinetic
and potential forms of low-degree polynomials (closed forms), the operator is symmetric,
and its harmonic-oscillator ground energy approaches the exact 3/2 with p."""
import numpy as np

from oracle import collocation as col
from oracle.mesh import Mesh

L = 6.0


def _mesh(p, n=3):
    br = np.linspace(-L, L, n + 1)
    return Mesh(br, br.copy(), br.copy(), p)


def test_kinetic_form_exact_for_quadratic_bubble():
    m = _mesh(4)
    X = m.node_coords()
    ub = np.prod(L ** 2 - X ** 2, axis=1) / m.minvsqrt
    k = np.vdot(ub, col.apply_H_gll(m, np.zeros(m.N_int), ub[None])[0]).real
    ref = 0.5 * 3 * (8 * L ** 3 / 3) * (16 * L ** 5 / 15) ** 2
    np.testing.assert_allclose(k, ref, rtol=1e-13)


def test_potential_form_is_the_gll_rule():
    m = _mesh(4)
    X = m.node_coords()
    u = np.prod(L ** 2 - X ** 2, axis=1)
    v = X[:, 0] ** 2 + 1.0
    ub = u / m.minvsqrt
    e = np.vdot(ub, col.apply_H_gll(m, v, ub[None])[0] - col.apply_H_gll(m, np.zeros(m.N_int), ub[None])[0]).real
    a2 = 16 * L ** 5 / 15                  # int (L^2 - x^2)^2
    a4 = 16 * L ** 7 / 105                 # int x^2 (L^2 - x^2)^2
    np.testing.assert_allclose(e, a4 * a2 * a2 + a2 ** 3, rtol=1e-13)


def test_symmetric():
    m = _mesh(3, 2)
    H = col.dense_Hbar_gll(m, np.random.default_rng(1).uniform(-1, 1, m.N_int))
    assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()


def test_harmonic_ground_energy_converges():
    errs = []
    for p in (4, 6):
        m = _mesh(p, 2)
        X = m.node_coords()
        v = 0.5 * np.sum(X ** 2, axis=1)
        lam = np.linalg.eigvalsh(col.dense_Hbar_gll(m, v))[0]
        errs.append(abs(lam - 1.5))
    assert errs[1] < 2e-2 and errs[1] < errs[0] / 5
