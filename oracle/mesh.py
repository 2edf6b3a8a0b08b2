"""Tensor-product hexahedral mesh with spectral (GLL) nodes (oracle).

Elements are the axis-aligned boxes [X_ex, X_ex+1] x [Y_ey, Y_ey+1] x [Z_ez, Z_ez+1];
each carries (p+1)^3 GLL nodes (Sec. VI.A).  Orbitals satisfy a homogeneous
Dirichlet condition on the domain boundary (Eq. 13), so the unknowns are the
interior nodes only.

Orderings used everywhere in the oracle:
  element      e = ex + nx*(ey + ny*ez)
  local node   l = a + (p+1)*(b + (p+1)*c)          (a along x fastest)
  quad point   q = qx + nq*(qy + nq*qz)
  full node    G = I + Nx*(J + Ny*K),  Nx = nx*p+1  (includes the boundary)
  interior     (I-1) + (Nx-2)*((J-1) + (Ny-2)*(K-1))

The overlap matrix M is integrated with the GLL rule on the nodes themselves,
so M is diagonal (Sec. VI.A): M_jj = sum over elements e containing node j of
J_e w_a w_b w_c with J_e = hx hy hz / 8.  This oracle builds it literally as
that sum over elements, with an explicit connectivity array.
"""
from __future__ import annotations

import numpy as np

from .basis import gauss, gll, lagrange_tables


class Mesh:
    def __init__(self, X, Y, Z, p: int, nq: int = 0):
        self.breaks = [np.asarray(X, float), np.asarray(Y, float), np.asarray(Z, float)]
        self.n = [len(b) - 1 for b in self.breaks]
        if min(self.n) < 1:
            raise ValueError("at least one element per axis")
        self.p = int(p)
        self.P1 = self.p + 1
        self.nq = int(nq) if nq else self.p + 1
        self.xi, self.w = gll(self.p)[:2]
        self.eta, self.omega = gauss(self.nq)[:2]
        self.B, self.D = lagrange_tables(self.p, self.nq)
        self.h = [np.diff(b) for b in self.breaks]
        if any((h <= 0).any() for h in self.h):
            raise ValueError("breakpoints must increase")
        self.Nn = [nd * self.p + 1 for nd in self.n]          # full nodes per axis
        self.Ni = [nn - 2 for nn in self.Nn]                   # interior nodes per axis
        self.n_elem = self.n[0] * self.n[1] * self.n[2]
        self.N_full = self.Nn[0] * self.Nn[1] * self.Nn[2]
        self.N_int = self.Ni[0] * self.Ni[1] * self.Ni[2]
        self._build_nodes()
        self._build_connectivity()
        self._build_mass()

    # ---- 1-D node coordinates per axis ------------------------------------
    def _build_nodes(self):
        self.axis_coords = []
        for d in range(3):
            b, h = self.breaks[d], self.h[d]
            c = np.zeros(self.Nn[d])
            for e in range(self.n[d]):
                for a in range(self.P1):
                    c[e * self.p + a] = b[e] + 0.5 * (self.xi[a] + 1.0) * h[e]
            c[-1] = b[-1]
            self.axis_coords.append(c)

    # ---- explicit element -> node connectivity ----------------------------
    def _build_connectivity(self):
        nx, ny, nz = self.n
        P1, p = self.P1, self.p
        Nx, Ny = self.Nn[0], self.Nn[1]
        conn = np.zeros((self.n_elem, P1 ** 3), dtype=np.int64)
        ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
        eidx = ex + nx * (ey + ny * ez)
        for c in range(P1):
            for b in range(P1):
                for a in range(P1):
                    loc = a + P1 * (b + P1 * c)
                    I = ex * p + a
                    J = ey * p + b
                    K = ez * p + c
                    conn[eidx, loc] = I + Nx * (J + Ny * K)
        self.conn = conn
        self.elem_xyz = np.zeros((self.n_elem, 3), dtype=np.int64)
        self.elem_xyz[eidx] = np.stack([ex, ey, ez], axis=1)
        hx = self.h[0][self.elem_xyz[:, 0]]
        hy = self.h[1][self.elem_xyz[:, 1]]
        hz = self.h[2][self.elem_xyz[:, 2]]
        self.elem_h = np.stack([hx, hy, hz], axis=1)
        self.jac = hx * hy * hz / 8.0                       # det of the affine map
        # interior mask and maps
        I, J, K = np.meshgrid(np.arange(self.Nn[0]), np.arange(self.Nn[1]),
                              np.arange(self.Nn[2]), indexing="ij")
        inner = ((I > 0) & (I < self.Nn[0] - 1) & (J > 0) & (J < self.Nn[1] - 1)
                 & (K > 0) & (K < self.Nn[2] - 1))
        full_of = (I + Nx * (J + Ny * K))
        int_of = (I - 1) + self.Ni[0] * ((J - 1) + self.Ni[1] * (K - 1))
        self.int_to_full = np.zeros(self.N_int, dtype=np.int64)
        self.int_to_full[int_of[inner]] = full_of[inner]
        self.full_to_int = -np.ones(self.N_full, dtype=np.int64)
        self.full_to_int[self.int_to_full] = np.arange(self.N_int)

    # ---- GLL-lumped overlap: sum over elements of J_e w_a w_b w_c ----------
    def _build_mass(self):
        wloc = np.kron(self.w, np.kron(self.w, self.w))      # [c,b,a] order
        contrib = self.jac[:, None] * wloc[None, :]
        Mfull = np.bincount(self.conn.ravel(), weights=contrib.ravel(), minlength=self.N_full)
        self.M = Mfull[self.int_to_full]
        self.minvsqrt = 1.0 / np.sqrt(self.M)

    # ---- coordinates -------------------------------------------------------
    def node_coords(self) -> np.ndarray:
        """(N_int, 3) coordinates of the interior nodes."""
        Nx, Ny = self.Nn[0], self.Nn[1]
        G = self.int_to_full
        I = G % Nx
        J = (G // Nx) % Ny
        K = G // (Nx * Ny)
        return np.stack([self.axis_coords[0][I], self.axis_coords[1][J],
                         self.axis_coords[2][K]], axis=1)

    def quad_coords(self) -> np.ndarray:
        """(n_elem, nq^3, 3) coordinates of the Gauss points of every element."""
        nq = self.nq
        out = np.zeros((self.n_elem, nq ** 3, 3))
        for d in range(3):
            lo = self.breaks[d][self.elem_xyz[:, d]]
            h = self.elem_h[:, d]
            pts = lo[:, None] + 0.5 * (self.eta[None, :] + 1.0) * h[:, None]  # (n_elem, nq)
            # broadcast to [qz, qy, qx]
            if d == 0:
                v = np.broadcast_to(pts[:, None, None, :], (self.n_elem, nq, nq, nq))
            elif d == 1:
                v = np.broadcast_to(pts[:, None, :, None], (self.n_elem, nq, nq, nq))
            else:
                v = np.broadcast_to(pts[:, :, None, None], (self.n_elem, nq, nq, nq))
            out[:, :, d] = v.reshape(self.n_elem, -1)
        return out

    def quad_weights(self) -> np.ndarray:
        """(n_elem, nq^3) Gauss weight times Jacobian: the measure of each point."""
        W = np.kron(self.omega, np.kron(self.omega, self.omega))
        return self.jac[:, None] * W[None, :]

    @classmethod
    def from_config(cls, cfg):
        return cls(cfg.X, cfg.Y, cfg.Z, cfg.p, cfg.nq)
