"""GLL-collocation variant of the discrete Hamiltonian (oracle).

Test infrastructure only (see oracle/__init__.py).

The paper integrates the overlap with the GLL rule on the element nodes (diagonal M)
and every other integral with the Gauss rule (Sec. VI.A).  This variant integrates the
Hamiltonian with the GLL rule as well (spectral-element collocation):
  * kinetic form 1/2 int grad N_j . grad N_k by the tensor GLL rule: per element
    sum_d c_d (K1g along d) (x) W (x) W with K1g = Dn^T W Dn (Dn: basis derivatives at the
    GLL nodes, W: GLL weights) and c_d = J (2/h_d)^2 / 2;
  * potential form int V N_j N_k by the GLL rule = M_jj V(x_j) delta_jk, so in the Loewdin
    basis (Eq. 21) the potential acts as the diagonal V(x_j).
Hbar_gll psibar = M^-1/2 K_gll M^-1/2 psibar + V(x_j) psibar_j.  The kinetic integrand is
not integrated exactly (degree 2p per axis against a rule exact to 2p - 1), so this is a
different operator from the paper's; its error against the Gauss form is a measured
quantity, not a parity target.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham
from .basis import gll_derivative
from .mesh import Mesh


def _kinetic_tables(p: int, w: np.ndarray):
    Dn = gll_derivative(p)
    I = np.eye(p + 1)
    G = (np.kron(I, np.kron(I, Dn)), np.kron(I, np.kron(Dn, I)), np.kron(Dn, np.kron(I, I)))
    W = np.kron(w, np.kron(w, w))
    return G, W


def apply_H_gll(mesh: Mesh, v_nodes: np.ndarray, psibar: np.ndarray) -> np.ndarray:
    """Hbar_gll psibar; v_nodes: V at the interior nodes (N_int); psibar (..., N_int)."""
    G, W = _kinetic_tables(mesh.p, mesh.w)
    psi = psibar * mesh.minvsqrt
    lead = psi.shape[:-1]
    psi2 = psi.reshape((-1, mesh.N_int))
    out = np.zeros_like(psi2, dtype=np.result_type(psi2, np.float64))
    wJ = mesh.jac[:, None] * W[None, :]
    for r in range(psi2.shape[0]):
        ue = ham.to_full(mesh, psi2[r])[mesh.conn]
        ye = 0.0
        for d in range(3):
            s2 = (2.0 / mesh.elem_h[:, d]) ** 2
            ye = ye + ((0.5 * s2[:, None] * wJ) * (ue @ G[d].T)) @ G[d]
        out[r] = ham._scatter(mesh, ye[None])[0][mesh.int_to_full]
    res = out * mesh.minvsqrt + psibar.reshape(psi2.shape) * v_nodes[None, :]
    return res.reshape(lead + (mesh.N_int,))


def dense_Hbar_gll(mesh: Mesh, v_nodes: np.ndarray) -> np.ndarray:
    I = np.eye(mesh.N_int)
    return apply_H_gll(mesh, v_nodes, I).T
