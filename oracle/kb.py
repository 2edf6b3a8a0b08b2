"""Nonlocal pseudopotential in the Kleinman-Bylander form (oracle).

Test infrastructure only (see oracle/__init__.py).

Eq. 6 (Sec. II): the nonlocal part acts as
    V_nl phi = sum_{I,l,m} [ int chi_Ilm phi / h_Ilm ] chi_Ilm,
    chi_Ilm = dV_l^I u_lm^I,   h_Ilm = int u_lm^I dV_l^I u_lm^I.
Its Galerkin matrix in the finite-element basis (Eq. 15) is
    H_nl[j, k] = sum_p P[j, p] P[k, p] / h_p,   P[j, p] = int chi_p N_j,
every integral by the tensor Gauss rule (Sec. VI.A), and in the Loewdin basis
(Eq. 21) Hbar_nl = M^-1/2 P D P^T M^-1/2 with D = diag(1 / h_p).  The
denominators h_p are integrated with the same Gauss rule.

Synthetic projectors (stand-ins for tabulated pseudopotential data): for an atom
at R, with d = r - R,
    u_lm(r)  = exp(-|d|^2 / (2 a^2)) Y_lm(d),  Y_00 = 1,  Y_1m = d_x, d_y, d_z,
    dV_l(r)  = c_l exp(-|d|^2 / (2 b^2)),
projectors ordered atom by atom, l = 0 then (for lmax = 1) d_x, d_y, d_z.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham
from .mesh import Mesh


def _harmonics(d: np.ndarray, lmax: int):
    """Real solid harmonics Y_lm(d) used by the projectors, in projector order."""
    out = [(0, np.ones(d.shape[:-1]))]
    if lmax >= 1:
        out += [(1, d[..., 0]), (1, d[..., 1]), (1, d[..., 2])]
    return out


class KleinmanBylander:
    """Projector data of a set of atoms on a mesh and the action of Hbar_nl."""

    def __init__(self, mesh: Mesh, R, a: float, b: float, c, lmax: int = 1):
        self.mesh = mesh
        R = np.atleast_2d(np.asarray(R, float))
        xq = mesh.quad_coords()
        wq = mesh.quad_weights()
        chis, hs = [], []
        for I in range(len(R)):
            d = xq - R[I][None, None, :]
            r2 = np.sum(d * d, axis=-1)
            gu = np.exp(-r2 / (2 * a * a))
            for l, Y in _harmonics(d, lmax):
                u = gu * Y
                dV = c[l] * np.exp(-r2 / (2 * b * b))
                chis.append(dV * u)
                hs.append(float(np.sum(wq * u * dV * u)))
        self.chi_q = np.array(chis)                   # (n_proj, n_elem, nq^3)
        self.h = np.array(hs)
        # P[:, p] = int chi_p N_j over the interior nodes (load vector of chi_p)
        self.P = np.stack([ham.load_vector(mesh, ch) for ch in self.chi_q], axis=1)
        self.n_proj = len(hs)

    def project(self, psibar: np.ndarray) -> np.ndarray:
        """C[p, a] = (P^T M^-1/2 psibar_a)_p = int chi_p psi_a."""
        psibar = np.atleast_2d(psibar)
        return self.P.T @ (psibar * self.mesh.minvsqrt[None, :]).T

    def apply(self, psibar: np.ndarray) -> np.ndarray:
        """Hbar_nl psibar = M^-1/2 P D P^T M^-1/2 psibar, orbital by orbital (same shape
        as psibar: one vector or a block [n_orb, N_int])."""
        C = self.project(psibar)
        y = (self.P @ (C / self.h[:, None])).T * self.mesh.minvsqrt[None, :]
        return y.reshape(np.shape(psibar))

    def dense(self) -> np.ndarray:
        Pb = self.P * self.mesh.minvsqrt[:, None]
        return Pb @ np.diag(1.0 / self.h) @ Pb.T
