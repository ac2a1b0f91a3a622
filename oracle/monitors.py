"""Convergence monitors of the flexible shifted solver (oracle).

Test infrastructure: imported by the tests only, never by the product path.

Followed passages (Section 3):
  Prop. 1, Eq. genritz: the Ritz pairs (theta, u = V_{m+1} H_bar_m f) of
      (K + sigma M) M^{-1} solve H_m(sigma; T_m) f = theta H_m f, with
      H_m(sigma; T_m) = I + H_m (sigma I - T_m) the square part of
      Eq. shiftedarnoldimod and H_m the square part of H_bar_m.
  Eq. residualritzeigen: their residual is
      -h_{m+1,m} v_{m+1} (tau_m + theta_k - sigma) e_m^* f_k, so
      rho_k = |h_{m+1,m}| |tau_m + theta_k - sigma| |e_m^* f_k| (||v_{m+1}|| = 1).
  Prop. 2, Eq. fomresidualineq: the FFOM residual is at most
      sum_k rho_k |(sigma - tau_m) / (theta_k + tau_m - sigma)| |theta_k^{-1}| |s_k|,
      s_k = e_k^* F^{-1} H_m^{-1} beta e_1.
  Prop. 3, Eq. fomgmresresdiff: ||r_fom - r_gmres|| <= alpha (1 + alpha) / (1 + alpha^2) ||r_fom||,
      alpha = ||eta H_m(sigma; T_m)^{-*} e_m||, eta = h_{m+1,m} (sigma - tau_m).

H is the (m+1) x m flexible Hessenberg matrix of Algorithm 3 (as in
oracle.fgmres, H[i, k] = h_{i+1,k+1}), taus the steps' preconditioner shifts.
Everything is complex128 and uses dense NumPy / SciPy linear algebra.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def square_shifted(H, taus, sigma, m):
    """H_m(sigma; T_m) = I + H_m (sigma I - T_m), m x m."""
    return np.eye(m, dtype=np.complex128) + H[:m, :m] * (sigma - np.asarray(taus[:m]))[None, :]


def ritz_pairs(H, taus, sigma, m):
    """(theta, F): the generalized eigenpairs of H_m(sigma; T_m) f = theta H_m f."""
    theta, F = sla.eig(square_shifted(H, taus, sigma, m), H[:m, :m].astype(np.complex128))
    return theta, F


def ritz_residual_norms(H, taus, sigma, m, theta, F):
    """rho_k of Eq. residualritzeigen for the eigenvectors as scaled in F."""
    return np.abs(H[m, m - 1]) * np.abs(taus[m - 1] + theta - sigma) * np.abs(F[m - 1, :])


def fom_residual_bound(H, taus, sigma, m, beta):
    """The right-hand side of Eq. fomresidualineq."""
    theta, F = ritz_pairs(H, taus, sigma, m)
    rho = ritz_residual_norms(H, taus, sigma, m, theta, F)
    e1 = np.zeros(m, dtype=np.complex128)
    e1[0] = beta
    s = np.linalg.solve(F, np.linalg.solve(H[:m, :m], e1))
    d = sigma - taus[m - 1]
    return float(np.sum(rho * np.abs(d / (theta + taus[m - 1] - sigma)) * np.abs(1.0 / theta) * np.abs(s)))


def gmres_alpha(H, taus, sigma, m):
    """alpha of Prop. 3 at step m."""
    eta = H[m, m - 1] * (sigma - taus[m - 1])
    em = np.zeros(m, dtype=np.complex128)
    em[m - 1] = 1.0
    w = np.linalg.solve(square_shifted(H, taus, sigma, m).conj().T, em)
    return float(abs(eta) * np.linalg.norm(w))
