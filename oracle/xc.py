"""Adiabatic LDA exchange-correlation potential (oracle).

Sec. II uses the ALDA in the Ceperley-Alder form.  The paper prints no
parametrization; this oracle uses the spin-unpolarized Perdew-Zunger fit to the
Ceperley-Alder data (Phys. Rev. B 23, 5048 (1981), Appendix C):

  r_s = (3 / (4 pi rho))^(1/3)
  e_x = -(3/4) (3/pi)^(1/3) rho^(1/3),            v_x = (4/3) e_x
  r_s >= 1: e_c = g / (1 + b1 sqrt(r_s) + b2 r_s)
            v_c = e_c (1 + 7/6 b1 sqrt(r_s) + 4/3 b2 r_s) / (1 + b1 sqrt(r_s) + b2 r_s)
  r_s <  1: e_c = A ln r_s + B + C r_s ln r_s + D r_s
            v_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2 D - C)/3 r_s
  g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116

v_xc = d(rho e_xc)/d rho.  Below rho = 1e-14 the potential is set to zero.
"""
from __future__ import annotations

import numpy as np

GAMMA, BETA1, BETA2 = -0.1423, 1.0529, 0.3334
A_, B_, C_, D_ = 0.0311, -0.048, 0.0020, -0.0116
RHO_FLOOR = 1e-14


def eps_xc(rho: np.ndarray) -> np.ndarray:
    """Exchange-correlation energy per electron."""
    rho = np.asarray(rho, float)
    out = np.zeros_like(rho)
    m = rho >= RHO_FLOOR
    r = rho[m]
    rs = (3.0 / (4.0 * np.pi * r)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * r ** (1.0 / 3.0)
    ec = np.where(rs >= 1.0,
                  GAMMA / (1.0 + BETA1 * np.sqrt(rs) + BETA2 * rs),
                  A_ * np.log(rs) + B_ + C_ * rs * np.log(rs) + D_ * rs)
    out[m] = ex + ec
    return out


def v_xc(rho: np.ndarray) -> np.ndarray:
    """Exchange-correlation potential d(rho e_xc)/d rho."""
    rho = np.asarray(rho, float)
    out = np.zeros_like(rho)
    m = rho >= RHO_FLOOR
    r = rho[m]
    rs = (3.0 / (4.0 * np.pi * r)) ** (1.0 / 3.0)
    vx = -(3.0 * r / np.pi) ** (1.0 / 3.0)
    sq = np.sqrt(rs)
    den = 1.0 + BETA1 * sq + BETA2 * rs
    vc_hi = (GAMMA / den) * (1.0 + (7.0 / 6.0) * BETA1 * sq + (4.0 / 3.0) * BETA2 * rs) / den
    lr = np.log(rs)
    vc_lo = A_ * lr + (B_ - A_ / 3.0) + (2.0 / 3.0) * C_ * rs * lr + (2.0 * D_ - C_) / 3.0 * rs
    out[m] = vx + np.where(rs >= 1.0, vc_hi, vc_lo)
    return out
