"""Pins for the oracle adjoint: LDA kernel by finite differences, the Frechet
term against scipy.linalg.expm_frechet, dot-product (transpose) tests of the density
and Hartree/LDA adjoints, and the full gradient against central finite differences
of the oracle's own forward propagation."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import adjoint
from oracle import hamiltonian as ham
from oracle.mesh import Mesh
from oracle.propagate import Propagator


def test_vxc_prime_is_derivative_of_vxc():
    from oracle import xc
    rho = np.logspace(-6, 2, 37)
    h = 1e-6 * rho
    fd = (xc.v_xc(rho + h) - xc.v_xc(rho - h)) / (2 * h)
    np.testing.assert_allclose(adjoint.vxc_prime(rho), fd, rtol=1e-6)


def test_frechet_term_matches_expm_frechet():
    m = Mesh(np.linspace(-1.5, 1.5, 4), np.linspace(-1, 1, 3), np.linspace(-1, 1, 3), 2)
    rng = np.random.default_rng(2)
    v = rng.uniform(-2, 1, size=(m.n_elem, m.nq ** 3))
    dv = rng.standard_normal(v.shape)
    psi = synth.random_psi(2, m.N_int, 3)
    lam = synth.random_psi(2, m.N_int, 4)
    tau = 0.4
    g = adjoint.frechet_v(m, v, psi, lam, tau, tol=1e-13, n_s=16)
    H = ham.dense_Hbar(m, v)
    dH = ham.dense_Hbar(m, v + dv) - H            # the potential form is linear in v
    L = scipy.linalg.expm_frechet(-1j * tau * H, -1j * tau * dH, compute_expm=False)
    ref = sum(np.vdot(lam[a], L @ psi[a]).real for a in range(2))
    assert abs(np.sum(g * dv) - ref) < 1e-9 * max(1.0, abs(ref))


@pytest.mark.parametrize("hartree", [True, False])
def test_gradient_matches_central_differences(hartree):
    cfg = synth.small_config(3, 2, 2, p=3, n_orb=2, hartree=hartree)
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=5)
    N, dt = 3, 0.1
    rng = np.random.default_rng(6)
    E = rng.uniform(-0.05, 0.05, size=(N, 2, 3))
    w = np.full(N + 1, dt)
    w[0] = w[-1] = 0.5 * dt
    e = np.array([0.2, -0.3, 0.93])
    mk = lambda: Propagator.from_config(cfg, m, tol=1e-13, k_max=200)
    J, g = adjoint.objective_and_gradient(mk(), psi0, E, w, e, dt, n_s=12)
    h = 1e-4
    fd = np.zeros_like(E)
    for idx in np.ndindex(E.shape):
        Ep, Em = E.copy(), E.copy()
        Ep[idx] += h
        Em[idx] -= h
        Jp = _J(mk(), psi0, Ep, w, e, dt)
        Jm = _J(mk(), psi0, Em, w, e, dt)
        fd[idx] = (Jp - Jm) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def _J(prop, psi0, E, w, e, dt):
    d0 = prop.init(psi0)
    J = w[0] * (e @ d0) ** 2
    psi = psi0
    for n in range(E.shape[0]):
        psi, d, _ = prop.magnus_step(psi, dt, E[n, 0], E[n, 1])
        J += w[n + 1] * (e @ d) ** 2
    return J


def _dot_mesh():
    return Mesh(np.linspace(-2.0, 2.0, 4), np.linspace(-1.5, 1.5, 3), np.linspace(-1.0, 1.5, 3), 3)


def test_density_adjoint_is_the_transpose_of_the_linearized_density():
    """Dot-product test: sum_q g_q drho_q = Re <lambda, dpsi> with lambda the density
    adjoint of g.  rho is quadratic in psi, so its central difference with step 1 is the
    exact linearization."""
    m = _dot_mesh()
    rng = np.random.default_rng(21)
    occ = np.array([2.0, 1.0])
    psi = synth.random_psi(2, m.N_int, 22)
    dpsi = synth.random_psi(2, m.N_int, 23)
    g = rng.standard_normal((m.n_elem, m.nq ** 3))
    drho = 0.5 * (ham.density(m, psi + dpsi, occ) - ham.density(m, psi - dpsi, occ))
    lam = adjoint.density_adjoint(m, psi, g, occ)
    lhs = np.sum(g * drho)
    rhs = sum(np.vdot(lam[a], dpsi[a]).real for a in range(2))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_hartree_adjoint_is_the_transpose_of_the_hartree_map():
    """Dot-product test of the Hartree part of the potential adjoint: V_H is linear in
    rho, so sum_q g_q V_H[drho]_q = sum_q hxc_adjoint(g)_q drho_q."""
    from oracle import poisson
    m = _dot_mesh()
    rng = np.random.default_rng(24)
    rho = np.abs(rng.standard_normal((m.n_elem, m.nq ** 3)))
    drho = rng.standard_normal(rho.shape)
    g = rng.standard_normal(rho.shape)
    dvh, _, _ = poisson.hartree(m, drho, None, 1e-14)
    gr = adjoint.hxc_adjoint(m, rho, g, hartree=True, use_xc=False)
    lhs, rhs = np.sum(g * dvh), np.sum(gr * drho)
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_xc_adjoint_is_the_linearized_lda_potential():
    """The LDA part of the potential adjoint against a central difference of v_xc itself."""
    from oracle import xc
    m = _dot_mesh()
    rng = np.random.default_rng(25)
    rho = rng.uniform(0.01, 2.0, size=(m.n_elem, m.nq ** 3))
    drho = rng.standard_normal(rho.shape)
    g = rng.standard_normal(rho.shape)
    eps = 1e-6
    dv = (xc.v_xc(rho + eps * drho) - xc.v_xc(rho - eps * drho)) / (2 * eps)
    gr = adjoint.hxc_adjoint(m, rho, g, hartree=False, use_xc=True)
    lhs, rhs = np.sum(g * dv), np.sum(gr * drho)
    assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs))
