"""Projected L-BFGS polish of a candidate (oracle).

The paper's DA method couples a global search with a local search (Sec. III-A);
the polish here plays that role after the swarm. The paper does not give a
local optimiser, so this is the textbook limited-memory BFGS (Nocedal and
Wright, Numerical Optimization, Alg. 7.4 two-loop recursion and Alg. 3.1
backtracking) with the iterate projected onto the box [lo, hi]^N:
  * history m = 8 pairs (s, y), stored only when s^T y > eps * y^T y;
  * initial inverse Hessian gamma I, gamma = s^T y / y^T y of the newest pair,
    or 1 / max(1, ||g||_inf) with no history;
  * a direction with g^T d >= 0 is replaced by -g / max(1, ||g||_inf) and the
    history is cleared;
  * trial points theta_t = clip(theta + 2^-t d, lo, hi), t = 0..19, the first one
    meeting Armijo f(theta_t) <= f + c1 g^T (theta_t - theta), c1 = 1e-4, is taken;
    if none does, the polish stops;
  * a fixed number of iterations (50).
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps


def two_loop(g, S, Y):
    """H g by the two-loop recursion over history pairs (oldest first in S, Y)."""
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / (y @ s)
        a = rho * (s @ q)
        q = q - a * y
        alphas.append(a)
    if S:
        gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    else:
        gamma = 1.0 / max(1.0, float(np.max(np.abs(g))))
    z = gamma * q
    for (s, y), a in zip(zip(S, Y), reversed(alphas)):
        rho = 1.0 / (y @ s)
        beta = rho * (y @ z)
        z = z + s * (a - beta)
    return z


def polish(cost_grad_fn, theta0, lo: float, hi: float, iters: int = 50, m: int = 8,
           c1: float = 1e-4, max_trials: int = 20):
    """Polish theta0 (N,). cost_grad_fn(theta) -> (cost, grad). Returns (theta, cost, n_evals)."""
    th = np.clip(np.asarray(theta0, np.float64), lo, hi)
    f, g = cost_grad_fn(th)
    S, Y = [], []
    n_evals = 1
    for _ in range(iters):
        d = -two_loop(g, S, Y)
        if not (g @ d < 0.0):
            d = -g / max(1.0, float(np.max(np.abs(g))))
            S, Y = [], []
        accepted = False
        for t in range(max_trials):
            tt = np.clip(th + (0.5 ** t) * d, lo, hi)
            ft, gt = cost_grad_fn(tt)
            n_evals += 1
            if ft <= f + c1 * (g @ (tt - th)):
                accepted = True
                break
        if not accepted:
            break
        s, y = tt - th, gt - g
        if s @ y > EPS * (y @ y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        th, f, g = tt, ft, gt
    return th, f, n_evals
