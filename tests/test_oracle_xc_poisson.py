"""Pins for the oracle's LDA (Sec. II, Perdew-Zunger fit) and Poisson solve (Eqs. 8a, 19)."""
import math

import numpy as np
import pytest

from oracle import hamiltonian as ham
from oracle import poisson, xc
from oracle.mesh import Mesh


def test_vxc_is_derivative_of_energy_density():
    rho = np.logspace(-6, 2, 41)
    h = 1e-6 * rho
    f = lambda r: r * xc.eps_xc(r)
    fd = (f(rho + h) - f(rho - h)) / (2 * h)
    np.testing.assert_allclose(xc.v_xc(rho), fd, rtol=1e-7)


def test_exchange_closed_form_and_floor():
    # e_x(r_s) = -(3/4)(9/(4 pi^2))^(1/3) / r_s = -0.4581652932831429 / r_s
    rs = 2.0
    rho = 3.0 / (4 * math.pi * rs ** 3)
    ex = -0.4581652932831429 / rs
    ec = -0.1423 / (1 + 1.0529 * math.sqrt(rs) + 0.3334 * rs)
    assert abs(xc.eps_xc(np.array([rho]))[0] - (ex + ec)) < 1e-14
    assert xc.v_xc(np.array([1e-15]))[0] == 0.0


def test_correlation_branches_continuous_at_rs_1():
    """The published fit joins its two branches at r_s = 1 to ~3e-5 Ha."""
    rho1 = 3.0 / (4 * math.pi)
    lo = xc.eps_xc(np.array([rho1 * (1 + 1e-9)]))[0]
    hi = xc.eps_xc(np.array([rho1 * (1 - 1e-9)]))[0]
    assert abs(lo - hi) < 5e-5
    vlo = xc.v_xc(np.array([rho1 * (1 + 1e-9)]))[0]
    vhi = xc.v_xc(np.array([rho1 * (1 - 1e-9)]))[0]
    assert abs(vlo - vhi) < 5e-5


@pytest.mark.parametrize("p", [2, 4])
def test_poisson_reproduces_polynomial_solution(p):
    """phi = prod (L^2 - x^2) lies in the FE space; with rho = -lap(phi)/(4 pi)
    exactly integrated, the Galerkin solution is phi itself."""
    Ls = np.array([2.0, 2.5, 3.0])
    br = [np.linspace(-Ls[d], Ls[d], n + 1) for d, n in enumerate((2, 3, 2))]
    m = Mesh(*br, p)
    xq = m.quad_coords()
    f = [Ls[d] ** 2 - xq[:, :, d] ** 2 for d in range(3)]
    lap = -2.0 * (f[1] * f[2] + f[0] * f[2] + f[0] * f[1])
    rho = -lap / (4 * math.pi)
    vq, phi, it = poisson.hartree(m, rho, tol=1e-14)
    X = m.node_coords()
    ex = np.prod([Ls[d] ** 2 - X[:, d] ** 2 for d in range(3)], axis=0)
    np.testing.assert_allclose(phi, ex, rtol=1e-10, atol=1e-10 * ex.max())
    np.testing.assert_allclose(vq, f[0] * f[1] * f[2], atol=1e-10 * ex.max())


def test_poisson_gaussian_charge_far_from_boundary():
    """A narrow Gaussian charge in a large grounded box: V_H - V_free is the
    (harmonic) image term, nearly constant near the centre; its variation is small."""
    b = np.linspace(-12, 12, 7)
    m = Mesh(b, b, b, 5)
    xq = m.quad_coords()
    r = np.sqrt(np.sum(xq ** 2, axis=-1))
    s = 1.0
    rho = (2 * math.pi * s * s) ** -1.5 * np.exp(-r * r / (2 * s * s))
    vq, _, _ = poisson.hartree(m, rho, tol=1e-12)
    from scipy.special import erf
    vfree = np.where(r > 0, erf(r / (math.sqrt(2) * s)) / np.where(r > 0, r, 1), 0)
    near = r < 3.0
    diff = (vq - vfree)[near]
    # the image potential of a unit charge in a cube of half-side 12 is about -0.08
    assert -0.15 < diff.mean() < -0.03
    assert diff.max() - diff.min() < 0.01
