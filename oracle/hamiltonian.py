"""Discrete operators of the semi-discrete TDKS system (oracle).

* Eq. 15: H_jk = 1/2 int grad N_j . grad N_k + int V_KS N_j N_k, every integral
  by the tensor Gauss rule (Sec. VI.A), evaluated element by element from the
  basis values and gradients at the Gauss points.
* Eq. 21: Hbar = M^-1/2 H M^-1/2 acting on psibar = M^1/2 psi.
* Eq. 2: rho = sum_a f_a |psi_a|^2 at the Gauss points.
* Eq. 19: K_jk = int grad N_j . grad N_k and c_j = int rho N_j.
* Sec. V (Eq. 30): dipole mu = int r rho, by the same Gauss rule.

The element basis values N_l(x_q) and gradients are dense (nq^3 x (p+1)^3)
matrices formed as Kronecker products of the 1-D Lagrange tables: the basis of
a hexahedral Lagrange element is by definition the tensor product of 1-D
Lagrange polynomials.  Nothing is sum-factorized.
"""
from __future__ import annotations

import functools

import numpy as np

from .mesh import Mesh


@functools.lru_cache(maxsize=None)
def _ref_tables(p: int, nq: int, Bkey, Dkey):
    B = np.array(Bkey).reshape(nq, p + 1)
    D = np.array(Dkey).reshape(nq, p + 1)
    Nval = np.kron(B, np.kron(B, B))        # rows [qz,qy,qx], cols [c,b,a]
    Gx = np.kron(B, np.kron(B, D))          # d/dxi along x (reference)
    Gy = np.kron(B, np.kron(D, B))
    Gz = np.kron(D, np.kron(B, B))
    return Nval, (Gx, Gy, Gz)


def ref_tables(mesh: Mesh):
    return _ref_tables(mesh.p, mesh.nq, tuple(mesh.B.ravel()), tuple(mesh.D.ravel()))


def to_full(mesh: Mesh, v_int: np.ndarray) -> np.ndarray:
    """Interior vector(s) -> full node grid with zero Dirichlet values."""
    shape = v_int.shape[:-1] + (mesh.N_full,)
    out = np.zeros(shape, dtype=v_int.dtype)
    out[..., mesh.int_to_full] = v_int
    return out


def _scatter(mesh: Mesh, ye: np.ndarray, conn=None) -> np.ndarray:
    """Sum element contributions (..., n_e, P1^3) into the full node grid."""
    conn = mesh.conn if conn is None else conn
    idx = conn.ravel()
    lead = ye.shape[:-2]
    flat = ye.reshape((-1,) + ye.shape[-2:])
    outs = []
    for r in range(flat.shape[0]):
        v = flat[r].ravel()
        if np.iscomplexobj(v):
            o = (np.bincount(idx, weights=v.real, minlength=mesh.N_full)
                 + 1j * np.bincount(idx, weights=v.imag, minlength=mesh.N_full))
        else:
            o = np.bincount(idx, weights=v, minlength=mesh.N_full)
        outs.append(o)
    return np.array(outs).reshape(lead + (mesh.N_full,))


def _element_H(mesh: Mesh, ue: np.ndarray, v_q, elems, kinetic_scale: float):
    """y_e = kinetic_scale * int grad N . grad u + int V N u on the listed elements.

    ue: (..., len(elems), P1^3) nodal values; v_q: (len(elems), nq^3) or None."""
    Nval, G = ref_tables(mesh)
    W = np.kron(mesh.omega, np.kron(mesh.omega, mesh.omega))
    wJ = mesh.jac[elems][:, None] * W[None, :]                   # (ne, nq^3)
    ye = 0.0
    for d in range(3):
        s2 = (2.0 / mesh.elem_h[elems, d]) ** 2                  # chain rule, squared
        gd = ue @ G[d].T                                         # reference gradient
        ye = ye + ((kinetic_scale * s2[:, None] * wJ) * gd) @ G[d]
    if v_q is not None:
        uq = ue @ Nval.T
        ye = ye + ((wJ * v_q) * uq) @ Nval
    return ye


def apply_H(mesh: Mesh, v_q: np.ndarray, psibar: np.ndarray) -> np.ndarray:
    """Hbar psibar (Eqs. 15, 21).  psibar: (..., N_int) complex; v_q: (n_elem, nq^3)."""
    psi = psibar * mesh.minvsqrt                                 # psi = M^-1/2 psibar
    lead = psi.shape[:-1]
    psi2 = psi.reshape((-1, mesh.N_int))
    out = np.zeros_like(psi2, dtype=np.result_type(psi2, np.float64))
    elems = np.arange(mesh.n_elem)
    for r in range(psi2.shape[0]):
        ue = to_full(mesh, psi2[r])[mesh.conn]
        ye = _element_H(mesh, ue, v_q, elems, 0.5)
        out[r] = _scatter(mesh, ye[None])[0][mesh.int_to_full]
    return (out * mesh.minvsqrt).reshape(lead + (mesh.N_int,))


def _elements_of_full_nodes(mesh: Mesh, full_nodes: np.ndarray) -> np.ndarray:
    """Indices of all elements whose closure contains any of the given nodes."""
    Nx, Ny = mesh.Nn[0], mesh.Nn[1]
    I = full_nodes % Nx
    J = (full_nodes // Nx) % Ny
    K = full_nodes // (Nx * Ny)
    sets = []
    for idx, nd in ((I, mesh.n[0]), (J, mesh.n[1]), (K, mesh.n[2])):
        cand = []
        for off in (0, 1):
            e = idx // mesh.p - off
            ok = (e >= 0) & (e < nd) & (idx >= e * mesh.p) & (idx <= (e + 1) * mesh.p)
            cand.append(np.where(ok, e, -1))
        sets.append(cand)
    out = set()
    for a in sets[0]:
        for b in sets[1]:
            for c in sets[2]:
                ok = (a >= 0) & (b >= 0) & (c >= 0)
                e = a + mesh.n[0] * (b + mesh.n[1] * c)
                out.update(e[ok].tolist())
    return np.array(sorted(out), dtype=np.int64)


def apply_H_rows(mesh: Mesh, v_q: np.ndarray, psibar: np.ndarray, rows: np.ndarray):
    """(Hbar psibar)[..., rows] computed from the elements touching those rows only."""
    rows = np.asarray(rows, dtype=np.int64)
    full_rows = mesh.int_to_full[rows]
    elems = _elements_of_full_nodes(mesh, full_rows)
    psi = psibar * mesh.minvsqrt
    lead = psi.shape[:-1]
    psi2 = psi.reshape((-1, mesh.N_int))
    out = np.zeros((psi2.shape[0], len(rows)), dtype=np.result_type(psi2, np.float64))
    conn = mesh.conn[elems]
    for r in range(psi2.shape[0]):
        ue = to_full(mesh, psi2[r])[conn]
        ye = _element_H(mesh, ue, v_q[elems], elems, 0.5)
        full = _scatter(mesh, ye[None], conn)[0]
        out[r] = full[full_rows]
    return (out * mesh.minvsqrt[rows]).reshape(lead + (len(rows),))


def dense_Hbar(mesh: Mesh, v_q: np.ndarray) -> np.ndarray:
    """Assemble Hbar column by column from apply_H on unit vectors (tiny meshes)."""
    E = np.eye(mesh.N_int)
    return apply_H(mesh, v_q, E).T


def stiffness_apply(mesh: Mesh, u_int: np.ndarray) -> np.ndarray:
    """K u with K_jk = int grad N_j . grad N_k over interior nodes (Eq. 19)."""
    ue = to_full(mesh, u_int)[mesh.conn]
    ye = _element_H(mesh, ue, None, np.arange(mesh.n_elem), 1.0)
    return _scatter(mesh, ye[None])[0][mesh.int_to_full]


def stiffness_diag(mesh: Mesh) -> np.ndarray:
    """Diagonal of K: element diagonals int |grad N_l|^2 summed over elements."""
    _, G = ref_tables(mesh)
    W = np.kron(mesh.omega, np.kron(mesh.omega, mesh.omega))
    wJ = mesh.jac[:, None] * W[None, :]
    de = 0.0
    for d in range(3):
        s2 = (2.0 / mesh.elem_h[:, d]) ** 2
        de = de + (s2[:, None] * wJ) @ (G[d] ** 2)              # sum_q wJ s2 (dN_l)^2
    return _scatter(mesh, de[None])[0][mesh.int_to_full]


def interp_q(mesh: Mesh, f_int: np.ndarray) -> np.ndarray:
    """Values at every Gauss point of the FE function with interior coefficients f."""
    Nval, _ = ref_tables(mesh)
    return to_full(mesh, f_int)[..., mesh.conn] @ Nval.T


def density(mesh: Mesh, psibar: np.ndarray, occ) -> np.ndarray:
    """rho(x_q) = sum_a f_a |psi_a(x_q)|^2 with psi = M^-1/2 psibar (Eq. 2)."""
    rho = np.zeros((mesh.n_elem, mesh.nq ** 3))
    for a in range(psibar.shape[0]):
        vq = interp_q(mesh, psibar[a] * mesh.minvsqrt)
        rho += occ[a] * (vq.real ** 2 + vq.imag ** 2)
    return rho


def load_vector(mesh: Mesh, rho_q: np.ndarray) -> np.ndarray:
    """c_j = int rho N_j over interior nodes (Eq. 19)."""
    Nval, _ = ref_tables(mesh)
    ye = (mesh.quad_weights() * rho_q) @ Nval
    return _scatter(mesh, ye[None])[0][mesh.int_to_full]


def dipole(mesh: Mesh, rho_q: np.ndarray) -> np.ndarray:
    """mu = int r rho(r) dr by the Gauss rule (Sec. V, Eq. 30)."""
    xq = mesh.quad_coords()
    wq = mesh.quad_weights()
    return np.array([np.sum(wq * rho_q * xq[:, :, d]) for d in range(3)])


def integrate_q(mesh: Mesh, f_q: np.ndarray) -> float:
    return float(np.sum(mesh.quad_weights() * f_q))
