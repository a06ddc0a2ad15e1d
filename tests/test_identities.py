"""Algebraic identities the CUDA path relies on, checked numerically in FP64 (no GPU).

* Partial fractions of two Debye columns: with c = 1/(1 + j w tau),
  re_i re_j + im_i im_j = (tau_i re_i + tau_j re_j) / (tau_i + tau_j), so the pole
  block of the Gram A^T A follows from the column sums S_i = sum_k re_i(k).
* The damped cost of any x is a quadratic in x: with M = G + lam diag G,
  ||A x - b||^2 + lam sum G_jj x_j^2 = b^T b - 2 x^T h + x^T M x.
* The squared form of the column sums: with x = w tau, re = 1/(1 + x^2),
  im = x re and u = x^2 re^2, h_i = sum re_i eps' + tau_i sum re_i (w eps''),
  d re/d theta = -2 ln10 u and d im/d theta = ln10 w tau (re - 2u) (theta = log10 tau).
"""
import numpy as np

import workloads as W
from oracle import dls, models


def test_partial_fraction_gram_from_column_sums():
    rs = np.random.default_rng(0)
    om = W.log_grid(1e5, 1e11, 700)
    for _ in range(20):
        N = int(rs.integers(2, 21))
        th = rs.uniform(-13, -5, N)
        th[1] = th[0] + rs.choice([0.0, 1e-9, 1e-3])     # equal and nearly equal relaxation times
        A = dls.basis(om, th)                            # stacked real rows over imaginary rows
        G = A.T @ A
        tau = 10.0 ** th
        S = G[0, 1:]                                     # sum_k re_i(k)
        np.testing.assert_allclose(np.diag(G)[1:], S, rtol=1e-13)
        Gp = (tau[:, None] * S[:, None] + tau[None, :] * S[None, :]) / (tau[:, None] + tau[None, :])
        np.testing.assert_allclose(G[1:, 1:], Gp, rtol=1e-12)
        assert G[0, 0] == om.size


def test_damped_cost_is_a_quadratic_in_the_weights():
    b = W.mixed_batch(S=3, seed=2, P=8, K_range=(40, 300), N_range=(2, 8))
    re, im = models.synthesize(b)
    rs = np.random.default_rng(1)
    lam = dls.LAM_SEARCH
    for s in range(b.S):
        a, c = b.offsets[s], b.offsets[s + 1]
        N = int(b.n_poles[s])
        A = dls.basis(b.omega[a:c], rs.uniform(-12, -6, N))
        y = dls.target(re[a:c], im[a:c])
        G, h = A.T @ A, A.T @ y
        M = G + lam * np.diag(np.diag(G))
        for _ in range(5):
            x = rs.normal(0, 5, N + 1)
            direct = np.sum((A @ x - y) ** 2) + lam * np.sum(np.diag(G) * x * x)
            assert abs(y @ y - 2 * x @ h + x @ M @ x - direct) <= 1e-10 * (y @ y + direct)


def test_squared_form_of_the_column_sums_and_their_derivatives():
    b = W.mixed_batch(S=4, seed=6, P=8, K_range=(50, 400), N_range=(2, 12))
    re_t, im_t = models.synthesize(b)
    rs = np.random.default_rng(3)
    for s in range(b.S):
        a, c = b.offsets[s], b.offsets[s + 1]
        om, e1, e2 = b.omega[a:c], re_t[a:c], im_t[a:c]
        N = int(b.n_poles[s])
        th = rs.uniform(-12, -6, N)
        A = dls.basis(om, th)                              # rows: eps' block, then eps'' block
        K = om.size
        h = A.T @ dls.target(e1, e2)
        tau = 10.0 ** th
        x2 = (om[:, None] * tau[None, :]) ** 2
        re = 1.0 / (1.0 + x2)
        u = x2 * re * re
        np.testing.assert_allclose(u, re * (1.0 - re), rtol=1e-12, atol=1e-15)   # 1 - re cancels for re ~ 1
        hs = (re * e1[:, None]).sum(0) + tau * (re * (om * e2)[:, None]).sum(0)
        np.testing.assert_allclose(hs, h[1:], rtol=1e-12)
        # derivatives in theta against central differences of the basis columns
        d = 1e-6
        Ap, Am = dls.basis(om, th + d), dls.basis(om, th - d)
        dre_fd = (Ap[:K, 1:] - Am[:K, 1:]) / (2 * d)
        dim_fd = (Ap[K:, 1:] - Am[K:, 1:]) / (2 * d)
        ln10 = np.log(10.0)
        np.testing.assert_allclose(-2 * ln10 * u, dre_fd, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(ln10 * om[:, None] * tau * (re - 2 * u), dim_fd, rtol=1e-6, atol=1e-9)
