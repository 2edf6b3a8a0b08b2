"""Second-order Magnus propagation of the TDKS orbitals (oracle).

Eqs. 25-26: psibar^n = exp(-i Dt Hbar[rho(t_{n-1} + Dt/2)]) psibar^{n-1}.
Sec. VI.B, predictor-corrector for the midpoint Hamiltonian:
  1. predict V_HXC(t_{n-1} + Dt/4) by linear extrapolation from the two previous
     steps, 1.25 V_HXC^{n-1} - 0.25 V_HXC^{n-2}  (first step: V_HXC^{-1} = V_HXC^0);
  2. psibar^{n-1/2} = exp(-i Dt/2 Hbar[predicted]) psibar^{n-1};
  3. V_HXC(t_{n-1} + Dt/2) from the density of psibar^{n-1/2};
  4. psibar^n = exp(-i Dt Hbar[corrected]) psibar^{n-1};
  5. V_HXC^n from psibar^n (next step's history) and the dipole of rho^n.
V_KS = V_N + V_H + V_XC + V_field (Eqs. 3, 16) at the Gauss points; the field is
V_field = -E(t) . r (Eq. 7), evaluated at t_{n-1} + Dt/4 (predictor) and
t_{n-1} + Dt/2 (corrector).  The nuclear potential is fixed in time.
The delta kick multiplies the ground state by exp(-i kappa r.d) (Sec. VII.A),
applied to the nodal coefficients.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import hamiltonian as ham
from . import poisson, xc
from .lanczos import expm_lanczos
from .mesh import Mesh


def nuclear_potential(mesh: Mesh, kind: str, R, Z, param) -> np.ndarray:
    """V_N at the Gauss points for the synthetic nuclei of the workloads."""
    xq = mesh.quad_coords()
    v = np.zeros(xq.shape[:2])
    R = np.atleast_2d(np.asarray(R, float))
    Z = np.atleast_1d(np.asarray(Z, float))
    if kind == "none":
        return v
    if kind == "harmonic":
        d = xq - R[0][None, None, :]
        return 0.5 * param * param * np.sum(d * d, axis=-1)
    for I in range(len(Z)):
        d = xq - R[I][None, None, :]
        r = np.sqrt(np.sum(d * d, axis=-1))
        if kind == "soft":
            v -= Z[I] / np.sqrt(r * r + param)
        elif kind == "bare":
            v -= Z[I] / r
        elif kind == "erf":
            with np.errstate(divide="ignore", invalid="ignore"):
                val = np.where(r > 0, erf(r / param) / np.where(r > 0, r, 1.0),
                               2.0 / (math.sqrt(math.pi) * param))
            v -= Z[I] * val
        else:
            raise ValueError(kind)
    return v


def kick(mesh: Mesh, psibar: np.ndarray, kappa: float, direction) -> np.ndarray:
    d = np.asarray(direction, float)
    s = mesh.node_coords() @ d
    return psibar * np.exp(-1j * kappa * s)[None, :]


class Propagator:
    def __init__(self, mesh: Mesh, v_nuc: np.ndarray, occ, hartree=True, use_xc=True,
                 cg_tol=1e-13, tol=1e-10, k_max=64, nl=None):
        self.mesh = mesh
        self.nl = nl            # optional nonlocal (Kleinman-Bylander) term, Eq. 6
        self.v_nuc = v_nuc
        self.occ = np.asarray(occ, float)
        self.hartree_on = hartree
        self.xc_on = use_xc
        self.cg_tol = cg_tol
        self.tol = tol
        self.k_max = k_max
        self.xq = mesh.quad_coords()
        self.phi = np.zeros(mesh.N_int)
        self.vhxc_1 = None      # V_HXC at t_{n-1}
        self.vhxc_2 = None      # V_HXC at t_{n-2}
        self.cg_iters = []

    @classmethod
    def from_config(cls, cfg, mesh=None, **kw):
        mesh = mesh or Mesh.from_config(cfg)
        vn = nuclear_potential(mesh, cfg.nuc_kind, cfg.atom_R, cfg.atom_Z, cfg.nuc_param)
        kw.setdefault("tol", cfg.tol)
        kw.setdefault("k_max", cfg.k_max)
        return cls(mesh, vn, cfg.occ, cfg.hartree, cfg.xc, **kw)

    def v_field(self, E) -> np.ndarray:
        E = np.asarray(E, float)
        return -(self.xq @ E)

    def v_hxc(self, psibar):
        rho = ham.density(self.mesh, psibar, self.occ)
        v = np.zeros_like(rho)
        if self.hartree_on:
            vh, self.phi, it = poisson.hartree(self.mesh, rho, self.phi, self.cg_tol)
            self.cg_iters.append(it)
            v += vh
        if self.xc_on:
            v += xc.v_xc(rho)
        return v, rho

    def init(self, psibar):
        v0, rho0 = self.v_hxc(psibar)
        self.vhxc_1 = v0
        self.vhxc_2 = v0
        return ham.dipole(self.mesh, rho0)

    def hbar(self, v_q):
        """x -> Hbar x with the local potential v_q (and the nonlocal term if set)."""
        if self.nl is None:
            return lambda x: ham.apply_H(self.mesh, v_q, x)
        return lambda x: ham.apply_H(self.mesh, v_q, x) + self.nl.apply(x)

    def expm(self, v_q, psibar, tau, k_fixed=None):
        return expm_lanczos(self.hbar(v_q), psibar, tau, self.tol, self.k_max, k_fixed=k_fixed)

    def magnus_step(self, psibar, dt, E_quarter=(0, 0, 0), E_half=(0, 0, 0),
                    k_fixed=None, record=False):
        """One predictor-corrector Magnus step; returns (psibar^n, dipole^n, info).
        With record=True, info also holds the step's intermediates (for the adjoint)."""
        v_pred = self.v_nuc + 1.25 * self.vhxc_1 - 0.25 * self.vhxc_2 + self.v_field(E_quarter)
        kf1 = None if k_fixed is None else k_fixed[0]
        kf2 = None if k_fixed is None else k_fixed[1]
        psi_half, info1 = self.expm(v_pred, psibar, 0.5 * dt, kf1)
        vhxc_half, _ = self.v_hxc(psi_half)
        v_mid = self.v_nuc + vhxc_half + self.v_field(E_half)
        psi_new, info2 = self.expm(v_mid, psibar, dt, kf2)
        vhxc_new, rho = self.v_hxc(psi_new)
        self.vhxc_2 = self.vhxc_1
        self.vhxc_1 = vhxc_new
        info = {"k_half": info1["k"], "k_full": info2["k"]}
        if record:
            info.update(psi_prev=psibar, psi_half=psi_half, psi_new=psi_new, v_pred=v_pred,
                        v_mid=v_mid, rho_half=ham.density(self.mesh, psi_half, self.occ),
                        rho_new=rho)
        return psi_new, ham.dipole(self.mesh, rho), info

    def magnus_step_sc(self, psibar, dt, E_half=(0, 0, 0), sc_tol=1e-10, max_iter=50):
        """The fully self-consistent midpoint step (Sec. VI.B, the approach before the
        predictor-corrector): (i) V_HXC(t + Dt/2) by linear extrapolation,
        1.5 V_HXC^{n-1} - 0.5 V_HXC^{n-2}; (ii) psibar^n = exp(-i Dt Hbar[V_mid]) psibar^{n-1}
        and V_HXC^n from it; (iii) V_mid <- (V_HXC^{n-1} + V_HXC^n) / 2; (iv) repeat (ii)-(iii)
        until max |change of V_mid| <= sc_tol.  Returns (psibar^n, dipole^n, iterations)."""
        v_mid = 1.5 * self.vhxc_1 - 0.5 * self.vhxc_2
        vf = self.v_field(E_half)
        for it in range(1, max_iter + 1):
            psi_new, _ = self.expm(self.v_nuc + v_mid + vf, psibar, dt)
            v_new, rho = self.v_hxc(psi_new)
            v_next = 0.5 * (self.vhxc_1 + v_new)
            delta = float(np.abs(v_next - v_mid).max())
            v_mid = v_next
            if delta <= sc_tol:
                break
        else:
            raise RuntimeError("self-consistent midpoint iteration did not converge")
        self.vhxc_2 = self.vhxc_1
        self.vhxc_1 = v_new
        return psi_new, ham.dipole(self.mesh, rho), it

    def energy(self, psibar, E=(0, 0, 0)):
        """Total energy sum_a f_a <psibar_a|T + V_N + V_field|psibar_a> + E_H + E_xc."""
        rho = ham.density(self.mesh, psibar, self.occ)
        vext = self.v_nuc + self.v_field(E)
        hpsi = self.hbar(vext)(psibar)
        e1 = float(np.sum(self.occ * np.einsum("an,an->a", psibar.conj(), hpsi).real))
        eh = 0.0
        if self.hartree_on:
            vh, _, _ = poisson.hartree(self.mesh, rho, None, 1e-14)
            eh = 0.5 * ham.integrate_q(self.mesh, rho * vh)
        exc = ham.integrate_q(self.mesh, rho * xc.eps_xc(rho)) if self.xc_on else 0.0
        return e1 + eh + exc
