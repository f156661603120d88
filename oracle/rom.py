"""Transfer function, Jacobian and the one-sided reduced model (float64).

Plain definitions (Sec. 3.1 and Sec. 3.3):
    X = A~^-1 B~,  Z = A~^-1 C~,
    Psi(0; p)            = C~^T X                      (Sec. 3.1)
    d Psi / d p_k        = -Z^T Delta_k X,  Delta_k = d A~ / d p_k
                         = diag(h^2 d mu / d p_k)       (eq. newjac; D is fixed,
                                                         so only the absorption
                                                         diagonal depends on p)
Reduced model (eq. newreduced, omega = 0):
    A~_r = V^T A~ V,  B~_r = V^T B~,  C~_r = V^T C~,
    Psi_r = C~_r^T A~_r^-1 B~_r,
    d Psi_r / d p_k = -Z_r^T (V^T Delta_k V) X_r,  X_r = A~_r^-1 B~_r,
                                                   Z_r = A~_r^-1 C~_r.
With D tracking mu (oracle/operator.py), B~ and C~ depend on p too; the
product rule on Psi = C~^T A~^-1 B~ gives
    d Psi / d p_k   = dC~_k^T X + Z^T dB~_k - Z^T dA~_k X,
    d Psi_r / d p_k = (V^T dC~_k)^T X_r + Z_r^T (V^T dB~_k)
                      - Z_r^T (V^T dA~_k V) X_r
(full_eval_general, rom_eval_general; with dB~ = dC~ = 0 and
dA~_k = diag(h^2 dmu_k) they are full_eval and rom_eval).
Layouts: Psi[d, s] (detector d, source s); J[k, d, s].
Parity: pinned by central finite differences of Psi (direct solves), by
source-detector reciprocity, by a dense projection and by the interpolation
theorem of Sec. 3.4.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .solvers import direct_solve


def full_eval(At, Bt, Ct, h, dmu=None, X=None, Z=None):
    """Psi and (optionally) J from direct solves of the full-order system."""
    X = direct_solve(At, Bt) if X is None else X
    Z = direct_solve(At, Ct) if Z is None else Z
    Psi = Ct.T @ X
    J = None
    if dmu is not None:
        J = np.stack([-(Z.T @ ((h * h * dmu[k])[:, None] * X)) for k in range(dmu.shape[0])])
    return Psi, J


def rom_eval(V, At, Bt, Ct, h, dmu=None):
    """Psi_r and J_r of the one-sided reduced model (eq. newreduced)."""
    Ar = V.T @ (At @ V)
    Br = V.T @ Bt
    Cr = V.T @ Ct
    cho = sla.cho_factor(Ar)
    Xr = sla.cho_solve(cho, Br)
    Zr = sla.cho_solve(cho, Cr)
    Psi = Cr.T @ Xr
    J = None
    if dmu is not None:
        J = np.stack([-(Zr.T @ (V.T @ ((h * h * dmu[k])[:, None] * V)) @ Xr)
                      for k in range(dmu.shape[0])])
    return Psi, J


def full_eval_general(At, Bt, Ct, dA=None, dB=None, dC=None):
    """Psi and J from direct solves, with per-parameter derivatives dA[k]
    (sparse), dB[k] (n x nsrc) and dC[k] (n x ndet)."""
    X = direct_solve(At, Bt)
    Z = direct_solve(At, Ct)
    Psi = Ct.T @ X
    J = None
    if dA is not None:
        J = np.stack([dC[k].T @ X + Z.T @ dB[k] - Z.T @ (dA[k] @ X) for k in range(len(dA))])
    return Psi, J


def rom_eval_general(V, At, Bt, Ct, dA=None, dB=None, dC=None):
    """Psi_r and J_r of the one-sided reduced model with p-dependent B~, C~
    (the arguments are those of full_eval_general at the point p)."""
    Ar = V.T @ (At @ V)
    Br = V.T @ Bt
    Cr = V.T @ Ct
    cho = sla.cho_factor(Ar)
    Xr = sla.cho_solve(cho, Br)
    Zr = sla.cho_solve(cho, Cr)
    Psi = Cr.T @ Xr
    J = None
    if dA is not None:
        J = np.stack([(V.T @ dC[k]).T @ Xr + Zr.T @ (V.T @ dB[k]) - Zr.T @ (V.T @ (dA[k] @ V)) @ Xr
                      for k in range(len(dA))])
    return Psi, J
