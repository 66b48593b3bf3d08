"""Linearised global least-squares track fit (test infrastructure, FP64 numpy).

Independent check of the Kalman oracle on short tracks without scattering.
The Kalman inward pass is, for a linear model, exactly the minimiser of
  sum_i r_i^T V_i^-1 r_i + (p_last - p_out)^T P0^-1 (p_last - p_out)
over the parameters at the innermost cluster, where p_last is the state
transported to the outermost cluster and (p_out, P0) the prior the inward
pass starts from (Fruhwirth 1987, the Kalman filter as recursive least
squares).  Here that objective is minimised by Gauss-Newton with a numerical
Jacobian, using its own helix model written in the angle form
  sin(phi(X)) = sin(phi0) + kappa (X - x0),  y = y0 - (cos phi - cos phi0)/kappa,
  z = z0 + tanlambda * (phi - phi0)/kappa,  kappa = -kB Bz q/pT,
which shares no code with the oracle's chord-form propagation.
"""
from __future__ import annotations

import numpy as np

KB = 0.299792458e-2


def transport(p0: np.ndarray, x0: float, X: float, bz: float) -> np.ndarray:
    """State (y, z, sinphi, tanlambda, q/pT) at plane X from the state at x0."""
    y0, z0, s0, t, w = p0
    kap = -KB * bz * w
    phi0 = np.arcsin(s0)
    s1 = s0 + kap * (X - x0)
    phi1 = np.arcsin(s1)
    if abs(kap * (X - x0)) < 1e-9:
        # straight-line limit (series in kappa to second order)
        dphi = phi1 - phi0
        c0 = np.cos(phi0)
        arc = (X - x0) / c0 if abs(dphi) < 1e-300 else dphi / kap
        y = y0 + np.tan(phi0) * (X - x0) if abs(dphi) < 1e-300 else y0 - (np.cos(phi1) - c0) / kap
    else:
        arc = (phi1 - phi0) / kap
        y = y0 - (np.cos(phi1) - np.cos(phi0)) / kap
    z = z0 + t * arc
    return np.array([y, z, s1, t, w])


def fit_inward(x, y, z, sy2, sz2, p_out, P0, bz: float, p_start=None, iters: int = 50):
    """Gauss-Newton minimum of the inward objective; returns (p_ref, cov_ref).

    x, y, z, sy2, sz2: clusters in ascending x; the parameters are the state at
    x[0]; the prior acts on the state transported to x[-1]."""
    x = np.asarray(x, float)
    L = np.diag(1.0 / np.sqrt(np.diag(P0)))  # P0 is diagonal here
    wy, wz = 1.0 / np.sqrt(np.asarray(sy2, float)), 1.0 / np.sqrt(np.asarray(sz2, float))

    def resid(p):
        pred = np.array([transport(p, x[0], X, bz) for X in x])
        r_meas = np.concatenate([(np.asarray(y) - pred[:, 0]) * wy, (np.asarray(z) - pred[:, 1]) * wz])
        r_prior = L @ (pred[-1] - p_out)
        return np.concatenate([r_meas, r_prior])

    def jac(p):
        # A = d resid / d p by central differences
        r0 = resid(p)
        A = np.empty((r0.shape[0], 5))
        for j in range(5):
            dp = np.zeros(5)
            dp[j] = steps[j]
            A[:, j] = (resid(p + dp) - resid(p - dp)) / (2 * steps[j])
        return r0, A

    p = np.array(p_start if p_start is not None else p_out, float)
    steps = np.array([1e-4, 1e-4, 1e-7, 1e-7, 1e-5])
    for _ in range(iters):
        r0, A = jac(p)
        step = -np.linalg.solve(A.T @ A, A.T @ r0)
        p = p + step
        if np.all(np.abs(step) <= 1e-14 * (1 + np.abs(p))):
            break
    _, A = jac(p)
    return p, np.linalg.inv(A.T @ A)


def fit_two_priors(x, y, z, sy2, sz2, s_first, P_first, s_last, P_last, bz: float, p_start=None, iters: int = 50,
                   k_ref: int = 0):
    """Gauss-Newton minimum of
      sum_i r_i^T V_i^-1 r_i + (p(x_0) - s_first)^T P_first^-1 (p(x_0) - s_first)
                             + (p(x_last) - s_last)^T P_last^-1 (p(x_last) - s_last)
    over the state at x[k_ref] (the objective of a two-filter smoother whose
    forward filter starts from (s_first, P_first) at the innermost cluster
    and whose backward filter starts from (s_last, P_last) at the outermost
    one; both priors diagonal); returns (p_ref, cov_ref) at x[k_ref]."""
    x = np.asarray(x, float)
    Lf = np.diag(1.0 / np.sqrt(np.diag(P_first)))
    Ll = np.diag(1.0 / np.sqrt(np.diag(P_last)))
    wy, wz = 1.0 / np.sqrt(np.asarray(sy2, float)), 1.0 / np.sqrt(np.asarray(sz2, float))
    s_first, s_last = np.asarray(s_first, float), np.asarray(s_last, float)

    def resid(p):
        pred = np.array([transport(p, x[k_ref], X, bz) for X in x])
        r_meas = np.concatenate([(np.asarray(y) - pred[:, 0]) * wy, (np.asarray(z) - pred[:, 1]) * wz])
        return np.concatenate([r_meas, Lf @ (pred[0] - s_first), Ll @ (pred[-1] - s_last)])

    steps = np.array([1e-4, 1e-4, 1e-7, 1e-7, 1e-5])

    def jac(p):
        r0 = resid(p)
        A = np.empty((r0.shape[0], 5))
        for j in range(5):
            dp = np.zeros(5)
            dp[j] = steps[j]
            A[:, j] = (resid(p + dp) - resid(p - dp)) / (2 * steps[j])
        return r0, A

    p = np.array(p_start if p_start is not None else s_first, float)
    for _ in range(iters):
        r0, A = jac(p)
        step = -np.linalg.solve(A.T @ A, A.T @ r0)
        p = p + step
        if np.all(np.abs(step) <= 1e-14 * (1 + np.abs(p))):
            break
    _, A = jac(p)
    return p, np.linalg.inv(A.T @ A)
