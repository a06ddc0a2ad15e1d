"""Analytic gradient of the DLS cost with respect to theta = log10(tau) (oracle, FP64).

Variable projection (Golub-Pereyra): the weights are a function of the
relaxation times, x(theta) = M^-1 h with M = A^T A + lam diag(A^T A) and
h = A^T b, and the cost is F(theta, x_hat(theta)) with
F(theta, y) = ||A y - b||^2 + lam sum_j G_jj y_j^2 and x_hat = S x the flipped
weights (S = diag(1, sign x_1, ..., sign x_N), Sec. III-B).

Chain rule, for pole i (basis column a_i, derivative a_i' = d a_i / d theta_i):
  partial F / partial theta_i at fixed y = -2 y_i a_i'^T r_hat + 2 lam y_i^2 a_i^T a_i'
  grad_y F = -2 g_hat,   g_hat = A^T r_hat - lam D^2 x_hat,  r_hat = b - A x_hat
  d x / d theta_i = M^-1 v_i,  v_i = e_i (a_i'^T r - 2 lam x_i a_i'^T a_i) - x_i A^T a_i',
                                r = b - A x
so with w = M^-1 S g_hat
  dcost/dtheta_i = -2 x_hat_i a_i'^T r_hat + 2 lam x_hat_i^2 a_i^T a_i'
                   - 2 w_i a_i'^T r + 4 lam w_i x_i a_i^T a_i' + 2 x_i (A w)^T a_i'.
Without a flip x_hat = x is the minimiser, g_hat = 0, w = 0, and the formula
reduces to the envelope-theorem form (the first two terms).

Basis derivatives with u = w_k tau_i and d u / d theta_i = u ln 10:
  d/dtheta [1/(1+u^2)] = -2 u^2 ln10 / (1+u^2)^2
  d/dtheta [u/(1+u^2)] = u (1-u^2) ln10 / (1+u^2)^2
"""
from __future__ import annotations

import math

import numpy as np

from . import dls

LN10 = math.log(10.0)


def basis_derivative(omega: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """dA/dtheta stacked like `dls.basis`: column i+1 holds d a_{i+1} / d theta_i;
    column 0 (eps_inf) is zero. Shape (..., 2K, N+1)."""
    omega = np.asarray(omega, np.float64)
    theta = np.asarray(theta, np.float64)
    u = omega[:, None] * (10.0 ** theta)[..., None, :]
    den = (1.0 + u * u) ** 2
    dre = -2.0 * u * u * LN10 / den
    dim = u * (1.0 - u * u) * LN10 / den
    lead = theta.shape[:-1]
    K = omega.shape[0]
    z = np.zeros(lead + (K, 1))
    return np.concatenate([np.concatenate([z, dre], -1), np.concatenate([z, dim], -1)], -2)


def cost_grad(omega, eps_re, eps_im, theta, lam: float = dls.LAM_SEARCH):
    """Cost and d cost / d theta for one candidate theta (N,)."""
    theta = np.asarray(theta, np.float64)
    A = dls.basis(omega, theta)
    dA = basis_derivative(omega, theta)
    b = dls.target(eps_re, eps_im)
    x = dls.damped_solve(A, b, lam)
    xh = dls.flip(x)
    s = np.where(np.arange(x.shape[0]) == 0, 1.0, np.where(x < 0.0, -1.0, 1.0))
    G = A.T @ A
    d2 = np.diag(G).copy()
    M = G + lam * np.diag(d2)
    rh = b - A @ xh
    r = b - A @ x
    cost = float(rh @ rh + lam * (d2 * xh * xh).sum())
    g_hat = A.T @ rh - lam * d2 * xh
    w = np.linalg.solve(M, s * g_hat)
    Aw = A @ w
    t_rh = dA.T @ rh
    t_aa = (A * dA).sum(axis=0)
    t_r = dA.T @ r
    t_aw = dA.T @ Aw
    g = (-2.0 * xh * t_rh + 2.0 * lam * xh * xh * t_aa
         - 2.0 * w * t_r + 4.0 * lam * w * x * t_aa + 2.0 * x * t_aw)
    return cost, g[1:]


def cost_grad_population(omega, eps_re, eps_im, thetas, lam: float = dls.LAM_SEARCH):
    """Costs (P,) and gradients (P, N) of a population, one candidate at a time."""
    thetas = np.asarray(thetas, np.float64)
    costs = np.empty(thetas.shape[0])
    grads = np.empty_like(thetas)
    for p in range(thetas.shape[0]):
        costs[p], grads[p] = cost_grad(omega, eps_re, eps_im, thetas[p], lam)
    return costs, grads
