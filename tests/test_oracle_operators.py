"""Pins for the oracle's discrete operators: M (GLL-lumped), H (Eq. 15), Hbar (Eq. 21),
density (Eq. 2), Poisson load vector and stiffness (Eq. 19), dipole (Eq. 30).

Polynomial test functions u = prod_d (L_d^2 - x_d^2) (or with an extra linear
factor) lie in the FE space for p >= 2 (p >= 3 for the cubic one) and vanish
on the boundary, so every quadrature-exact integral is a closed form."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial as P

from oracle import hamiltonian as ham
from oracle.mesh import Mesh

L = np.array([3.0, 2.5, 2.0])


def _graded(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, size=n)
    return np.concatenate([[lo], lo + (hi - lo) * np.cumsum(w) / w.sum()])


def _mesh(p, graded=False, n=(3, 2, 2)):
    if graded:
        br = [_graded(-L[d], L[d], n[d], 10 + d) for d in range(3)]
    else:
        br = [np.linspace(-L[d], L[d], n[d] + 1) for d in range(3)]
    return Mesh(br[0], br[1], br[2], p)


def _bubble_polys(shift=0.0):
    """1-D factors (L^2 - x^2), optionally times (x + shift) along x."""
    fs = [P([L[d] ** 2, 0.0, -1.0]) for d in range(3)]
    if shift:
        fs[0] = fs[0] * P([shift, 1.0])
    return fs


def _integral(poly, d):
    q = poly.integ()
    return q(L[d]) - q(-L[d])


def _nodal(mesh, fs):
    X = mesh.node_coords()
    return fs[0](X[:, 0]) * fs[1](X[:, 1]) * fs[2](X[:, 2])


@pytest.mark.parametrize("graded", [False, True])
@pytest.mark.parametrize("p", [3, 4, 6])
def test_mass_closed_form(p, graded):
    m = _mesh(p, graded)
    fs = _bubble_polys()
    u = _nodal(m, fs)
    exact = np.prod([_integral(fs[d] ** 2, d) for d in range(3)])
    assert abs(u @ (m.M * u) - exact) <= 1e-12 * exact


@pytest.mark.parametrize("graded", [False, True])
@pytest.mark.parametrize("p", [2, 4, 5])
def test_kinetic_and_constant_potential_closed_form(p, graded):
    m = _mesh(p, graded)
    fs = _bubble_polys()
    u = _nodal(m, fs)
    psibar = np.sqrt(m.M) * u
    c = 0.37
    v = np.full((m.n_elem, m.nq ** 3), c)
    Hu = ham.apply_H(m, v, psibar.astype(complex))
    got = np.vdot(psibar, Hu).real
    grad2 = 0.0
    for d in range(3):
        t = 1.0
        for e in range(3):
            t *= _integral(fs[e].deriv() ** 2 if e == d else fs[e] ** 2, e)
        grad2 += t
    u2 = np.prod([_integral(fs[d] ** 2, d) for d in range(3)])     # Gauss rule is exact here
    exact = 0.5 * grad2 + c * u2
    assert abs(got - exact) <= 1e-12 * abs(exact)


@pytest.mark.parametrize("p", [3, 4])
def test_polynomial_potential_term_closed_form(p):
    """int V u^2 with V = x^2 - 2 y + 0.5 z (Gauss exact for nq = p+1 >= 4)."""
    m = _mesh(p)
    fs = _bubble_polys()
    u = _nodal(m, fs)
    xq = m.quad_coords()
    v = xq[:, :, 0] ** 2 - 2 * xq[:, :, 1] + 0.5 * xq[:, :, 2]
    psibar = (np.sqrt(m.M) * u).astype(complex)
    vzero = np.zeros_like(v)
    got = np.vdot(psibar, ham.apply_H(m, v, psibar) - ham.apply_H(m, vzero, psibar)).real
    u2 = [_integral(fs[d] ** 2, d) for d in range(3)]
    ex = (_integral(P([0, 0, 1]) * fs[0] ** 2, 0) * u2[1] * u2[2]
          - 2 * u2[0] * _integral(P([0, 1]) * fs[1] ** 2, 1) * u2[2]
          + 0.5 * u2[0] * u2[1] * _integral(P([0, 1]) * fs[2] ** 2, 2))
    assert abs(got - ex) <= 1e-11 * max(1.0, abs(ex))


def test_hbar_hermitian_and_real_symmetric():
    m = Mesh(np.linspace(-1, 1, 3), np.linspace(-1, 1, 3), np.linspace(-1, 1, 3), 2)
    rng = np.random.default_rng(3)
    v = rng.uniform(-2, 1, size=(m.n_elem, m.nq ** 3))
    H = ham.dense_Hbar(m, v)
    assert H.shape == (27, 27)
    assert np.abs(H - H.conj().T).max() <= 1e-14 * np.abs(H).max()
    assert np.abs(H.imag).max() == 0.0


def test_harmonic_oscillator_ground_energy():
    """V = r^2/2: lowest eigenvalue of Hbar -> 3/2 (spectral convergence)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    b = np.linspace(-7, 7, 5)
    m = Mesh(b, b, b, 6)
    xq = m.quad_coords()
    v = 0.5 * np.sum(xq ** 2, axis=-1)
    op = LinearOperator((m.N_int, m.N_int), dtype=float,
                        matvec=lambda x: ham.apply_H(m, v, np.asarray(x).ravel()).real)
    vals = eigsh(op, k=1, which="SA", tol=1e-12)[0]
    assert abs(vals[0] - 1.5) < 3e-4


def test_box_ground_energy():
    """V = 0 on a Dirichlet box of side a: lowest eigenvalue 3 pi^2 / (2 a^2)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    a = 4.0
    b = np.linspace(0, a, 3)
    m = Mesh(b, b, b, 6)
    v = np.zeros((m.n_elem, m.nq ** 3))
    op = LinearOperator((m.N_int, m.N_int), dtype=float,
                        matvec=lambda x: ham.apply_H(m, v, np.asarray(x).ravel()).real)
    vals = eigsh(op, k=1, which="SA", tol=1e-13)[0]
    assert abs(vals[0] - 3 * np.pi ** 2 / (2 * a * a)) < 1e-6


def test_apply_rows_matches_full():
    m = _mesh(4, graded=True)
    rng = np.random.default_rng(5)
    v = rng.uniform(-2, 1, size=(m.n_elem, m.nq ** 3))
    psi = rng.standard_normal((2, m.N_int)) + 1j * rng.standard_normal((2, m.N_int))
    full = ham.apply_H(m, v, psi)
    rows = rng.choice(m.N_int, size=40, replace=False)
    part = ham.apply_H_rows(m, v, psi, rows)
    np.testing.assert_allclose(part, full[:, rows], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("graded", [False, True])
def test_density_dipole_load_stiffness_closed_forms(graded):
    p = 4
    m = _mesh(p, graded)
    fs = _bubble_polys(shift=0.7)          # cubic in x: in the space for p >= 3
    u = _nodal(m, fs)
    psibar = (np.sqrt(m.M) * u)[None, :].astype(complex) * np.exp(0.3j)
    rho = ham.density(m, psibar, [2.0])
    xq = m.quad_coords()
    uq = fs[0](xq[:, :, 0]) * fs[1](xq[:, :, 1]) * fs[2](xq[:, :, 2])
    np.testing.assert_allclose(rho, 2.0 * uq ** 2, rtol=1e-12, atol=1e-12)
    # dipole: int x_d 2 u^2 (degree <= 8 per direction; Gauss with 5 points is exact to 9)
    u2 = [_integral(fs[d] ** 2, d) for d in range(3)]
    dip = ham.dipole(m, rho)
    scale = 2.0 * np.prod(u2) * L.max()
    for d in range(3):
        ex = 2.0 * np.prod([_integral(P([0, 1]) * fs[e] ** 2, e) if e == d else u2[e]
                            for e in range(3)])
        assert abs(dip[d] - ex) <= 1e-13 * scale
    # load vector tested against a second FE function g: c^T g = int rho g
    gs = _bubble_polys()
    g = _nodal(m, gs)
    c = ham.load_vector(m, rho)
    ex = 2.0 * np.prod([_integral(fs[d] ** 2 * gs[d], d) for d in range(3)])
    assert abs(c @ g - ex) <= 1e-11 * abs(ex)
    # stiffness: g^T K g = int |grad g|^2
    Kg = ham.stiffness_apply(m, g)
    grad2 = 0.0
    for d in range(3):
        t = 1.0
        for e in range(3):
            t *= _integral(gs[e].deriv() ** 2 if e == d else gs[e] ** 2, e)
        grad2 += t
    assert abs(g @ Kg - grad2) <= 1e-12 * grad2


def test_stiffness_diag_matches_dense():
    m = Mesh(np.linspace(-1, 1, 3), np.linspace(-1, 2, 4), np.linspace(0, 1, 2), 3)
    E = np.eye(m.N_int)
    K = np.array([ham.stiffness_apply(m, E[i]) for i in range(m.N_int)])
    np.testing.assert_allclose(ham.stiffness_diag(m), np.diag(K), rtol=1e-13)
    np.testing.assert_allclose(K, K.T, atol=1e-13 * np.abs(K).max())
