"""Self-consistent Kohn-Sham ground state, the initial state of Sec. VII (oracle).

The paper computes ground states with Chebyshev-filtered subspace iteration
(Sec. VII) and does not print its mixing scheme.  This oracle takes a fixed
number of SCF iterations: the lowest n_orb eigenvectors of the real symmetric
Hbar[V_N + V_H[rho_in] + V_XC[rho_in]] (ARPACK Lanczos), a new density, and
linear density mixing rho_in <- (1 - a) rho_in + a rho_out.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh

from . import hamiltonian as ham
from . import poisson, xc


def lowest_states(mesh, v_q, n_orb, v0=None, tol=1e-12):
    op = LinearOperator((mesh.N_int, mesh.N_int), dtype=float,
                        matvec=lambda x: ham.apply_H(mesh, v_q, np.asarray(x).ravel()).real)
    vals, vecs = eigsh(op, k=n_orb, which="SA", tol=tol, v0=v0, ncv=max(2 * n_orb + 1, 20))
    order = np.argsort(vals)
    return vals[order], vecs[:, order].T


def scf(mesh, v_nuc, occ, n_orb, n_iter=50, mix=0.5, hartree=True, use_xc=True):
    """Return (orbitals psibar (n_orb, N_int) real, eigenvalues, rho_in)."""
    occ = np.asarray(occ, float)
    vals, psi = lowest_states(mesh, v_nuc, n_orb)
    rho_in = ham.density(mesh, psi, occ)
    phi = None
    for _ in range(n_iter):
        v = v_nuc.copy()
        if hartree:
            vh, phi, _ = poisson.hartree(mesh, rho_in, phi, 1e-13)
            v += vh
        if use_xc:
            v += xc.v_xc(rho_in)
        vals, psi = lowest_states(mesh, v, n_orb, v0=psi[0])
        rho_out = ham.density(mesh, psi, occ)
        rho_in = (1.0 - mix) * rho_in + mix * rho_out
    return psi, vals, rho_in
