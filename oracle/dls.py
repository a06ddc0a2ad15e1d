"""Damped least-squares cost of a candidate relaxation-time set (oracle, FP64).

The fitting method (Sec. III-B) is hybrid: a global optimiser proposes the
relaxation times, and for each proposal the weights eps_inf and d_eps_n of the
multi-Debye expansion (Eq. 7), which enter linearly, are found by damped
least squares ("DLS", Sec. III-A). Negative weights get their sign flipped,
which worsens the fit and so penalises the proposal (Sec. III-B); the misfit
includes both the real and the imaginary part (Sec. III-B).

Readings where the paper is silent:
  * search variable theta_n = log10(tau_n);
  * damping: Marquardt scaling, i.e. minimise ||A x - b||^2 + lam * sum_j G_jj x_j^2
    with G = A^T A, solved by Householder QR of the scaled, augmented matrix
    [A D^-1; sqrt(lam) I] (D = diag of the column norms);
  * flip: x_hat_n = |x_n| for the d_eps entries (eps_inf is not flipped), and the
    cost is evaluated at x_hat: ||A x_hat - b||^2 + lam * sum_j G_jj x_hat_j^2;
  * norm: squared 2-norm over the stacked real and imaginary rows, unweighted.
"""
from __future__ import annotations

import numpy as np

LAM_SEARCH = 1e-3
# The reported weights are the DLS weights of the found relaxation times, at the
# same damping as the search (an undamped re-solve can turn a nearly repeated
# pole pair into huge opposite weights that the sign flip then penalises).
LAM_FINAL = LAM_SEARCH


def basis(omega: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Stacked real basis of Eq. 7 at tau_n = 10**theta_n.

    omega: (K,); theta: (..., N). Returns A with shape (..., 2K, N+1):
      rows 0..K-1  (matched to eps'):  [1, Re 1/(1 + j w_k tau_n)]
      rows K..2K-1 (matched to eps''): [0, -Im 1/(1 + j w_k tau_n)]
    """
    omega = np.asarray(omega, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    tau = 10.0 ** theta
    c = 1.0 / (1.0 + 1j * omega[:, None] * tau[..., None, :])   # (..., K, N)
    K = omega.shape[0]
    lead = theta.shape[:-1]
    ones = np.ones(lead + (K, 1))
    zeros = np.zeros(lead + (K, 1))
    top = np.concatenate([ones, c.real], axis=-1)
    bot = np.concatenate([zeros, -c.imag], axis=-1)
    return np.concatenate([top, bot], axis=-2)


def target(eps_re: np.ndarray, eps_im: np.ndarray) -> np.ndarray:
    """Right-hand side b = (eps'; eps'') stacked like the basis rows."""
    return np.concatenate([np.asarray(eps_re, np.float64), np.asarray(eps_im, np.float64)])


def damped_solve(A: np.ndarray, b: np.ndarray, lam: float) -> np.ndarray:
    """Weights x minimising ||A x - b||^2 + lam * sum_j ||A_j||^2 x_j^2.

    Householder QR (LAPACK geqrf via numpy) of [A D^-1; sqrt(lam) I] with
    D = diag(||A_j||), then x = D^-1 z. A: (..., M, n); b: (M,).
    """
    n = A.shape[-1]
    d = np.sqrt((A * A).sum(axis=-2))                     # (..., n)
    As = A / d[..., None, :]
    eye = np.broadcast_to(np.sqrt(lam) * np.eye(n), A.shape[:-2] + (n, n))
    aug = np.concatenate([As, eye], axis=-2)
    baug = np.concatenate([b, np.zeros(n)])
    Q, R = np.linalg.qr(aug)
    qtb = np.einsum("...mi,m->...i", Q, baug)
    z = np.linalg.solve(R, qtb[..., None])[..., 0]
    return z / d


def flip(x: np.ndarray) -> np.ndarray:
    """Sign flip of negative d_eps weights (Sec. III-B); eps_inf (index 0) is kept."""
    xh = np.array(x, dtype=np.float64, copy=True)
    xh[..., 1:] = np.abs(xh[..., 1:])
    return xh


def cost_at(A: np.ndarray, b: np.ndarray, x: np.ndarray, lam: float) -> np.ndarray:
    """||A x - b||^2 + lam * sum_j ||A_j||^2 x_j^2 (the damped objective at x)."""
    r = np.einsum("...mi,...i->...m", A, x) - b
    g_diag = (A * A).sum(axis=-2)
    return (r * r).sum(axis=-1) + lam * (g_diag * x * x).sum(axis=-1)


def cost(omega, eps_re, eps_im, theta, lam: float = LAM_SEARCH, return_weights: bool = False):
    """DLS cost of candidate(s) theta (..., N): damped solve, sign flip, misfit.

    Returns cost (...) and, if requested, the flipped weights x_hat (..., N+1)
    = (eps_inf, d_eps_1..N).
    """
    A = basis(omega, theta)
    b = target(eps_re, eps_im)
    x = damped_solve(A, b, lam)
    xh = flip(x)
    c = cost_at(A, b, xh, lam)
    return (c, xh) if return_weights else c


def cost_population(omega, eps_re, eps_im, thetas, lam: float = LAM_SEARCH, chunk: int = 256):
    """Costs and flipped weights of a population thetas (P, N), evaluated in chunks."""
    thetas = np.asarray(thetas, dtype=np.float64)
    P = thetas.shape[0]
    costs = np.empty(P)
    weights = np.empty((P, thetas.shape[1] + 1))
    for a in range(0, P, chunk):
        c, w = cost(omega, eps_re, eps_im, thetas[a:a + chunk], lam, return_weights=True)
        costs[a:a + chunk] = c
        weights[a:a + chunk] = w
    return costs, weights


def model_eps(omega, weights, theta) -> np.ndarray:
    """Complex multi-Debye permittivity (Eq. 7) of weights (eps_inf, d_eps) at tau = 10**theta."""
    tau = 10.0 ** np.asarray(theta, np.float64)
    w = np.asarray(weights, np.float64)
    return w[0] + (w[1:][None, :] / (1.0 + 1j * np.asarray(omega)[:, None] * tau[None, :])).sum(axis=1)


def avg_fractional_error(omega, eps_re, eps_im, weights, theta) -> float:
    """Average fractional error in percent (Sec. IV): mean relative error of eps'
    plus mean relative error of eps'', summed."""
    e = model_eps(omega, weights, theta)
    fr, fi = e.real, -e.imag
    er = np.mean(np.abs(fr - eps_re) / np.abs(eps_re))
    ei = np.mean(np.abs(fi - eps_im) / np.abs(eps_im))
    return 100.0 * (er + ei)


def rel_rms(eps_a: np.ndarray, eps_b: np.ndarray) -> float:
    """||eps_a - eps_b||_2 / ||eps_b||_2 over complex values."""
    return float(np.linalg.norm(eps_a - eps_b) / np.linalg.norm(eps_b))
