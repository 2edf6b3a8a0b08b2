"""Pins for the oracle's Kleinman-Bylander nonlocal term (Eq. 6 in the Galerkin,
Loewdin form): Gaussian integrals in closed form for the denominators h_p and the
projections int chi_p psi of polynomial FE functions, the expectation value
sum_p (int chi_p psi)^2 / h_p, symmetry and rank of Hbar_nl, and the Lanczos
exponential of Hbar + Hbar_nl against a dense matrix exponential."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import hamiltonian as ham
from oracle.kb import KleinmanBylander
from oracle.lanczos import expm_lanczos
from oracle.mesh import Mesh

L, A, B, C = 6.0, 1.0, 0.8, (-2.0, -1.0)
KH = 1 / A ** 2 + 1 / (2 * B ** 2)            # exponent of u dV u
KC = 1 / (2 * A ** 2) + 1 / (2 * B ** 2)      # exponent of chi = dV u
G0 = np.sqrt(np.pi / KC)
I1 = L ** 2 * G0 - G0 / (2 * KC)              # int (L^2 - x^2) exp(-KC x^2) dx
I2 = L ** 2 * G0 / (2 * KC) - 3 * G0 / (4 * KC ** 2)   # int x^2 (L^2 - x^2) exp(-KC x^2) dx


@pytest.fixture(scope="module")
def fine():
    br = np.linspace(-L, L, 13)
    m = Mesh(br, br.copy(), br.copy(), 6)
    return m, KleinmanBylander(m, [[0.0, 0.0, 0.0]], A, B, C, lmax=1)


def test_denominators_closed_form(fine):
    _, kb = fine
    h0 = C[0] * (np.pi / KH) ** 1.5
    h1 = C[1] * (np.pi / KH) ** 1.5 / (2 * KH)
    assert kb.n_proj == 4
    np.testing.assert_allclose(kb.h, [h0, h1, h1, h1], rtol=2e-9)


def test_projections_of_polynomials_closed_form(fine):
    m, kb = fine
    X = m.node_coords()
    phi = np.prod(L ** 2 - X ** 2, axis=1)      # in the FE space, zero on the boundary
    c_even = kb.project(phi / m.minvsqrt)[:, 0]
    c_odd = kb.project(phi * X[:, 0] / m.minvsqrt)[:, 0]
    np.testing.assert_allclose(c_even[0], C[0] * I1 ** 3, rtol=2e-9)
    np.testing.assert_allclose(c_odd[1], C[1] * I2 * I1 ** 2, rtol=2e-9)
    # parity: the odd function has no s or y/z components, the even one no p components
    assert abs(c_odd[0]) + abs(c_odd[2]) + abs(c_odd[3]) < 1e-11 * abs(c_odd[1])
    assert np.abs(c_even[1:]).max() < 1e-11 * abs(c_even[0])


def test_expectation_value_closed_form(fine):
    m, kb = fine
    X = m.node_coords()
    psib = (np.prod(L ** 2 - X ** 2, axis=1) / m.minvsqrt)[None, :]
    e = np.vdot(psib[0], kb.apply(psib)[0])
    h0 = C[0] * (np.pi / KH) ** 1.5
    np.testing.assert_allclose(e.real, (C[0] * I1 ** 3) ** 2 / h0, rtol=5e-9)
    assert abs(e.imag) < 1e-12 * abs(e.real)


def test_dense_operator_symmetric_and_rank():
    cfg = synth.small_config(2, 2, 2, p=3, n_orb=1)
    m = Mesh.from_config(cfg)
    kb = KleinmanBylander(m, [[0.3, -0.2, 0.1], [-1.5, 1.0, 0.5]], A, B, C, lmax=1)
    H = kb.dense()
    assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()
    assert np.linalg.matrix_rank(H, tol=1e-10 * np.abs(H).max()) == 8
    psi = synth.random_psi(2, m.N_int, 3)
    np.testing.assert_allclose(kb.apply(psi), (H @ psi.T).T, atol=1e-13 * np.abs(H).max())


def test_lanczos_with_nonlocal_term_matches_dense_expm():
    cfg = synth.small_config(2, 2, 2, p=3, n_orb=1)
    m = Mesh.from_config(cfg)
    kb = KleinmanBylander(m, [[0.3, -0.2, 0.1]], A, B, C, lmax=1)
    v = synth.random_potential(m.n_elem * m.nq ** 3, 5).reshape(m.n_elem, -1)
    Hd = ham.dense_Hbar(m, v) + kb.dense()
    psi = synth.random_psi(2, m.N_int, 4)
    out, _ = expm_lanczos(lambda x: ham.apply_H(m, v, x) + kb.apply(x), psi, 0.3, 1e-12, 200)
    ref = (scipy.linalg.expm(-0.3j * Hd) @ psi.T).T
    assert np.abs(out - ref).max() < 1e-10
