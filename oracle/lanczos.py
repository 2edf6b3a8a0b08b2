"""Adaptive Lanczos approximation of exp(-i tau Hbar) psibar (oracle).

Sec. VI.B, Eqs. 36-38.  For each orbital separately:
  q_1 = psibar / ||psibar||;  for j = 1, 2, ...:
    w = Hbar q_j;  alpha_j = Re(q_j^H w);  w -= alpha_j q_j + beta_{j-1} q_{j-1}
    beta_j = ||w||;  T_j = tridiag(beta, alpha, beta)  (Hbar Hermitian -> T real)
    y = exp(-i tau T_j) e_1                 (eigendecomposition of T_j, Eq. 37)
    eps_j = |tau| beta_j ||psibar|| |y_j|    (Eq. 38: the (j+1, j) entry of the
                                            projected -i tau Hbar has modulus |tau| beta_j;
                                            tau < 0 gives the backward propagator)
    stop when eps_j <= tol:  z = ||psibar|| Q_j y;  otherwise q_{j+1} = w / beta_j.
The plain three-term recurrence is the default (the paper names no
re-orthogonalization); full re-orthogonalization by classical Gram-Schmidt applied
twice is an option.

The paper sets no cap on the Krylov dimension.  With a cap k_max, an unconverged
basis is used for the largest sub-step tau' = tau_rem / 2^m (m = 1, 2, ...) whose
estimate eps(tau') <= tol; psibar advances by exp(-i tau' Hbar) and the
recurrence restarts for the remaining time.  This is the same operator: the
exponential of a fixed matrix composes exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


class NotConverged(RuntimeError):
    pass


def exp_tridiag_e1(alpha, beta_off, tau):
    """y = exp(-i tau T) e_1 for the real symmetric tridiagonal T (diag alpha,
    off-diagonal beta_off), via T = S diag(lam) S^T (LAPACK stemr/stebz)."""
    alpha = np.asarray(alpha, float)
    if len(alpha) == 1:
        return np.array([np.exp(-1j * tau * alpha[0])])
    lam, S = scipy.linalg.eigh_tridiagonal(alpha, np.asarray(beta_off, float))
    return S @ (np.exp(-1j * tau * lam) * S[0, :])


def expm_lanczos(apply_vec, psi: np.ndarray, tau: float, tol: float, k_max: int = 64,
                 max_sub: int = 1000, k_fixed=None, reorth: bool = False):
    """Return (exp(-i tau Hbar) psi, info).  psi: (n_orb, N) complex.

    info["k"][a] lists the Krylov dimension of every sub-step of orbital a.
    k_fixed (int or per-orbital sequence) forces the dimension of a single step
    (used to replay another implementation's stopping index).
    reorth: after the three-term update, w is orthogonalized against every basis
    vector so far by classical Gram-Schmidt applied twice (CGS2); alpha_j keeps its
    three-term value and beta_j = ||w|| is taken after the two passes."""
    psi = np.atleast_2d(psi)
    out = np.empty_like(psi, dtype=complex)
    info = {"k": [], "err": []}
    for a in range(psi.shape[0]):
        kf = None
        if k_fixed is not None:
            kf = int(k_fixed) if np.isscalar(k_fixed) else int(k_fixed[a])
        v = psi[a].astype(complex)
        t_rem = float(tau)
        ks, errs = [], []
        while t_rem != 0.0:
            if len(ks) >= max_sub:
                raise NotConverged(f"orbital {a}: more than {max_sub} sub-steps")
            nrm = np.linalg.norm(v)
            if nrm == 0.0:
                break
            Q = [v / nrm]
            alpha, beta = [], []
            done = False
            for j in range(k_max):
                w = apply_vec(Q[j])
                a_j = float(np.vdot(Q[j], w).real)
                w = w - a_j * Q[j]
                if j > 0:
                    w = w - beta[j - 1] * Q[j - 1]
                if reorth:
                    Qm = np.array(Q)                     # (j+1, N)
                    for _ in range(2):
                        w = w - Qm.T @ (Qm.conj() @ w)
                b_j = float(np.linalg.norm(w))
                alpha.append(a_j)
                beta.append(b_j)
                y = exp_tridiag_e1(alpha, beta[:-1], t_rem)
                err = abs(t_rem) * b_j * nrm * abs(y[-1])
                stop = (err <= tol) if kf is None else (j + 1 == kf)
                if stop or b_j == 0.0:
                    v = nrm * (np.array(Q).T @ y)
                    t_rem = 0.0
                    ks.append(j + 1)
                    errs.append(err)
                    done = True
                    break
                Q.append(w / b_j)
            if done:
                break
            if kf is not None:
                raise NotConverged("k_fixed larger than k_max")
            # sub-step with the basis of dimension k_max
            for m in range(1, 64):
                ts = t_rem / 2.0 ** m
                y = exp_tridiag_e1(alpha, beta[:-1], ts)
                err = abs(ts) * beta[-1] * nrm * abs(y[-1])
                if err <= tol:
                    break
            else:
                raise NotConverged("no admissible sub-step")
            v = nrm * (np.array(Q[:k_max]).T @ y)
            t_rem -= ts
            ks.append(k_max)
            errs.append(err)
        out[a] = v
        info["k"].append(ks)
        info["err"].append(errs)
    return out, info
