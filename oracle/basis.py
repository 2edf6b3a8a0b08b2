"""1-D node sets, quadrature rules and Lagrange tables (oracle).

Sec. VI.A: spectral elements place their nodes at the Gauss-Legendre-Lobatto
(GLL) points -- the end points and the roots of P_p' -- and the overlap matrix is
integrated with the GLL rule on those same points, which makes it diagonal.
All other integrals use the Gauss-Legendre rule.  An n-point GLL rule is exact
to degree 2n-3, an n-point Gauss rule to degree 2n-1.

Computed in 50-digit arithmetic (mpmath) and rounded once to float64.
"""
from __future__ import annotations

import functools

import mpmath as mp
import numpy as np

_DPS = 50


def _legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (x strictly inside (-1,1)
    for the derivative formula)."""
    p0, p1 = mp.mpf(1), x
    if n == 0:
        return p0, mp.mpf(0)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    dp = n * (p0 - x * p1) / (1 - x * x)
    return p1, dp


@functools.lru_cache(maxsize=None)
def gll(p: int):
    """GLL nodes (ascending) and weights for degree p (p+1 points)."""
    if p < 1:
        raise ValueError("p >= 1")
    with mp.workdps(_DPS):
        nodes = [mp.mpf(-1)]
        for i in range(1, p):
            x = -mp.cos(mp.pi * i / p)
            for _ in range(100):
                P, dP = _legendre(p, x)
                # P_p'' from Legendre's equation (1-x^2)P'' - 2xP' + p(p+1)P = 0
                d2P = (2 * x * dP - p * (p + 1) * P) / (1 - x * x)
                step = dP / d2P
                x -= step
                if abs(step) < mp.mpf(10) ** (-_DPS + 5):
                    break
            nodes.append(x)
        nodes.append(mp.mpf(1))
        weights = []
        for x in nodes:
            if abs(x) == 1:
                P = mp.mpf(1) if x > 0 else mp.mpf((-1) ** p)
            else:
                P, _ = _legendre(p, x)
            weights.append(mp.mpf(2) / (p * (p + 1) * P * P))
        return (np.array([float(v) for v in nodes]), np.array([float(v) for v in weights]),
                nodes, weights)


@functools.lru_cache(maxsize=None)
def gauss(n: int):
    """Gauss-Legendre points (ascending) and weights, n points."""
    if n < 1:
        raise ValueError("n >= 1")
    with mp.workdps(_DPS):
        pts = []
        for i in range(1, n + 1):
            x = -mp.cos(mp.pi * (i - mp.mpf(1) / 4) / (n + mp.mpf(1) / 2))
            for _ in range(100):
                P, dP = _legendre(n, x)
                step = P / dP
                x -= step
                if abs(step) < mp.mpf(10) ** (-_DPS + 5):
                    break
            pts.append(x)
        wts = []
        for x in pts:
            _, dP = _legendre(n, x)
            wts.append(mp.mpf(2) / ((1 - x * x) * dP * dP))
        return (np.array([float(v) for v in pts]), np.array([float(v) for v in wts]), pts, wts)


@functools.lru_cache(maxsize=None)
def lagrange_tables(p: int, nq: int):
    """B[q][i] = l_i(eta_q) and D[q][i] = l_i'(eta_q) for the GLL Lagrange basis
    l_0..l_p evaluated at the nq Gauss points (reference element [-1, 1])."""
    _, _, xi, _ = gll(p)
    _, _, eta, _ = gauss(nq)
    B = np.zeros((nq, p + 1))
    D = np.zeros((nq, p + 1))
    with mp.workdps(_DPS):
        for q in range(nq):
            x = eta[q]
            for i in range(p + 1):
                val = mp.mpf(1)
                for m in range(p + 1):
                    if m != i:
                        val *= (x - xi[m]) / (xi[i] - xi[m])
                der = mp.mpf(0)
                for l in range(p + 1):
                    if l == i:
                        continue
                    term = 1 / (xi[i] - xi[l])
                    for m in range(p + 1):
                        if m != i and m != l:
                            term *= (x - xi[m]) / (xi[i] - xi[m])
                    der += term
                B[q, i] = float(val)
                D[q, i] = float(der)
    return B, D


@functools.lru_cache(maxsize=None)
def gll_derivative(p: int):
    """Dn[q][i] = l_i'(xi_q): derivatives of the GLL Lagrange basis at the GLL nodes
    themselves (the basis values there are the identity)."""
    _, _, xi, _ = gll(p)
    Dn = np.zeros((p + 1, p + 1))
    with mp.workdps(_DPS):
        for q in range(p + 1):
            x = xi[q]
            for i in range(p + 1):
                der = mp.mpf(0)
                for l in range(p + 1):
                    if l == i:
                        continue
                    term = 1 / (xi[i] - xi[l])
                    for m in range(p + 1):
                        if m != i and m != l:
                            term *= (x - xi[m]) / (xi[i] - xi[m])
                    der += term
                Dn[q, i] = float(der)
    return Dn
