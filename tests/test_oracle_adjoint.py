"""Pins for the oracle adjoint: LDA kernel by finite differences, the Frechet
term against scipy.linalg.expm_frechet, and the full gradient against central
finite differences of the oracle's own forward propagation."""
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
