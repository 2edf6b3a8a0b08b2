"""Hartree potential from the discrete Poisson problem (oracle).

Eq. 8a recast as the FE system of Eq. 19, K phi_H = 4 pi c, with
K_jk = int grad N_j . grad N_k and c_j = int rho N_j.  The boundary value is
zero (homogeneous Dirichlet); V_H at the Gauss points is then the FE
interpolant sum_j N_j phi_j.  Solved by conjugate gradients with the Jacobi
(diagonal) preconditioner, stopping at ||r|| <= tol ||b||; the paper does not
name its solver.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as ham
from .mesh import Mesh


def pcg(apply_A, b, diag, x0=None, tol=1e-13, maxit=20000):
    """Preconditioned CG (textbook, Golub & Van Loan Alg. 11.5.1).  Returns (x, iters)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0
    r = b - apply_A(x)
    if np.linalg.norm(r) <= tol * bnorm:
        return x, 0
    z = r / diag
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = apply_A(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        if np.linalg.norm(r) <= tol * bnorm:
            return x, it
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise RuntimeError("PCG did not converge")


def hartree(mesh: Mesh, rho_q: np.ndarray, phi0=None, tol=1e-13):
    """Return (V_H at the Gauss points, phi_H at the interior nodes, CG iterations)."""
    b = 4.0 * np.pi * ham.load_vector(mesh, rho_q)
    diag = ham.stiffness_diag(mesh)
    phi, it = pcg(lambda u: ham.stiffness_apply(mesh, u), b, diag, phi0, tol)
    return ham.interp_q(mesh, phi), phi, it
