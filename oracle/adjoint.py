"""Adjoint (reverse-mode gradient) of the Magnus predictor-corrector propagation (oracle).

Objective: J = sum_n w_n (e . mu(t_n))^2 over the dipoles of Sec. V after each step,
as a function of the field samples E(t_{n-1} + Dt/4), E(t_{n-1} + Dt/2) that enter
V_field = -E . r (Eq. 7) in the predictor and the corrector (Sec. VI.B).

Reverse sweep through one step (notation of propagate.py):
  psi' = U(v_mid) psi,  psi_h = U_h(v_pred) psi,  U(v) = exp(-i tau Hbar[v])  (Eq. 25)
  * adjoint propagation: lambda <- U^H lambda' = exp(+i tau Hbar) lambda' (Hbar Hermitian);
  * potential term (Frechet derivative of the exponential):
      dU psi = int_0^1 e^{-i tau (1-s) Hbar} (-i tau dHbar) e^{-i tau s Hbar} psi ds, so
      dJ/dv(x_q) = tau wJ_q int_0^1 sum_a Im[conj(mu_s(x_q)) phi_s(x_q)] ds,
      phi_s = e^{-i tau s Hbar} psi, mu_s = e^{+i tau (1-s) Hbar} lambda'
    (the potential form of Eq. 15 is int v conj(a) b), s by Gauss-Legendre;
  * V_H = interp K^-1 4 pi load(rho) (Eq. 19) with K symmetric:
      dJ/drho = 4 pi wJ . interp(K^-1 (B^T)^(x)3 dJ/dV_H);
  * LDA: dJ/drho += v_xc'(rho) dJ/dV_XC;
  * density rho = sum_a f_a |psi_a(x_q)|^2:  lambda_a += 2 f_a M^-1/2 (B^T)^(x)3 (dJ/drho psi_a(x_q)).
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham
from . import poisson
from .lanczos import expm_lanczos
from .xc import A_, B_, BETA1, BETA2, C_, D_, GAMMA, RHO_FLOOR


def vxc_prime(rho: np.ndarray) -> np.ndarray:
    """d v_xc / d rho of the Perdew-Zunger LDA (0 below the density floor)."""
    rho = np.asarray(rho, float)
    out = np.zeros_like(rho)
    m = rho >= RHO_FLOOR
    r = rho[m]
    rs = (3.0 / (4.0 * np.pi * r)) ** (1.0 / 3.0)
    dvx = -(1.0 / 3.0) * (3.0 / np.pi) ** (1.0 / 3.0) * r ** (-2.0 / 3.0)
    sq = np.sqrt(rs)
    Dn = 1.0 + BETA1 * sq + BETA2 * rs
    Nn = 1.0 + (7.0 / 6.0) * BETA1 * sq + (4.0 / 3.0) * BETA2 * rs
    dD = 0.5 * BETA1 / sq + BETA2
    dN = (7.0 / 12.0) * BETA1 / sq + (4.0 / 3.0) * BETA2
    dvc_hi = GAMMA * (dN * Dn - 2.0 * Nn * dD) / Dn ** 3
    dvc_lo = A_ / rs + (2.0 / 3.0) * C_ * (np.log(rs) + 1.0) + (2.0 * D_ - C_) / 3.0
    dvc_drs = np.where(rs >= 1.0, dvc_hi, dvc_lo)
    out[m] = dvx + dvc_drs * (-rs / (3.0 * r))
    return out


def hxc_adjoint(mesh, rho, g_h, hartree=True, use_xc=True):
    """dJ/drho at the Gauss points from dJ/dV_HXC there."""
    g = np.zeros_like(rho)
    wq = mesh.quad_weights()
    if hartree:
        y = ham.load_vector(mesh, g_h / wq)                 # (B^T)^(x)3 g_h, assembled
        z, _ = poisson.pcg(lambda u: ham.stiffness_apply(mesh, u), y, ham.stiffness_diag(mesh),
                           None, 1e-14)
        g += 4.0 * np.pi * wq * ham.interp_q(mesh, z)
    if use_xc:
        g += vxc_prime(rho) * g_h
    return g


def density_adjoint(mesh, psi, g_rho, occ):
    """lambda_a = 2 f_a M^-1/2 (B^T)^(x)3 (g_rho psi_a(x_q)) for every orbital."""
    wq = mesh.quad_weights()
    lam = np.zeros_like(psi, dtype=complex)
    for a in range(psi.shape[0]):
        pq = ham.interp_q(mesh, psi[a] * mesh.minvsqrt)
        lam[a] = 2.0 * occ[a] * mesh.minvsqrt * ham.load_vector(mesh, g_rho * pq / wq)
    return lam


def gauss_legendre_01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def frechet_v(mesh, v_q, psi, lam, tau, tol=1e-12, k_max=200, n_s=12, nl=None):
    """dJ/dv(x_q) of Re<lam, exp(-i tau Hbar[v]) psi> (summed over orbitals); nl: an
    optional v-independent nonlocal term of Hbar."""
    if nl is None:
        H = lambda x: ham.apply_H(mesh, v_q, x)
    else:
        H = lambda x: ham.apply_H(mesh, v_q, x) + nl.apply(x)
    wq = mesh.quad_weights()
    g = np.zeros((mesh.n_elem, mesh.nq ** 3))
    for s, ws in zip(*gauss_legendre_01(n_s)):
        phi, _ = expm_lanczos(H, psi, tau * s, tol, k_max)
        mu, _ = expm_lanczos(H, lam, -tau * (1.0 - s), tol, k_max)
        for a in range(psi.shape[0]):
            pq = ham.interp_q(mesh, phi[a] * mesh.minvsqrt)
            mq = ham.interp_q(mesh, mu[a] * mesh.minvsqrt)
            g += ws * tau * np.imag(np.conj(mq) * pq)
    return g * wq


def objective_and_gradient(prop, psi0, E, w, e, dt, n_s=12, tol_adj=1e-12):
    """J = sum_n w_n (e . mu_n)^2 and dJ/dE (shape (N, 2, 3): field at t+Dt/4, t+Dt/2).

    prop: a fresh Propagator; psi0: initial orbitals; E: (N, 2, 3); w: (N+1,)."""
    mesh = prop.mesh
    E = np.asarray(E, float)
    e = np.asarray(e, float)
    N = E.shape[0]
    d0 = prop.init(psi0)
    J = w[0] * (e @ d0) ** 2
    recs = []
    psi = psi0
    for n in range(N):
        psi, d, info = prop.magnus_step(psi, dt, E[n, 0], E[n, 1], record=True)
        info["d"] = d
        recs.append(info)
        J += w[n + 1] * (e @ d) ** 2
    xq = mesh.quad_coords()
    wq = mesh.quad_weights()
    ex = xq @ e
    H = prop.hbar
    lam = np.zeros_like(psi0, dtype=complex)
    gh1 = np.zeros((mesh.n_elem, mesh.nq ** 3))
    gh2 = np.zeros_like(gh1)
    dJdE = np.zeros_like(E)
    hb, xcb = prop.hartree_on, prop.xc_on
    for n in reversed(range(N)):
        r = recs[n]
        g_rho = hxc_adjoint(mesh, r["rho_new"], gh1, hb, xcb) + 2.0 * w[n + 1] * (e @ r["d"]) * wq * ex
        lam = lam + density_adjoint(mesh, r["psi_new"], g_rho, prop.occ)
        gh1_next = gh2.copy()
        g_vmid = frechet_v(mesh, r["v_mid"], r["psi_prev"], lam, dt, tol_adj, n_s=n_s, nl=prop.nl)
        lam_prev, _ = expm_lanczos(H(r["v_mid"]), lam, -dt, tol_adj, 200)
        dJdE[n, 1] = -np.einsum("eq,eqd->d", g_vmid, xq)
        lam_h = density_adjoint(mesh, r["psi_half"], hxc_adjoint(mesh, r["rho_half"], g_vmid, hb, xcb),
                                prop.occ)
        g_vpred = frechet_v(mesh, r["v_pred"], r["psi_prev"], lam_h, 0.5 * dt, tol_adj, n_s=n_s,
                            nl=prop.nl)
        lam_prev = lam_prev + expm_lanczos(H(r["v_pred"]), lam_h, -0.5 * dt, tol_adj, 200)[0]
        dJdE[n, 0] = -np.einsum("eq,eqd->d", g_vpred, xq)
        gh1 = gh1_next + 1.25 * g_vpred
        gh2 = -0.25 * g_vpred
        lam = lam_prev
    return J, dJdE
