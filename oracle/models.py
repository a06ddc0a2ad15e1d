"""Target permittivity models (oracle, FP64, test infrastructure only).

All functions return the complex relative permittivity eps(omega) following the
paper's sign convention eps = eps' - j eps'' (Eq. 1), so that a lossy material
has eps'' = -Im(eps) >= 0. `split` turns a complex array into (eps', eps'').
Complex powers use numpy's principal branch.
"""
from __future__ import annotations

import math

import numpy as np

import workloads as W


def split(eps: np.ndarray):
    """(eps', eps'') from complex eps = eps' - j eps'' (Eq. 1)."""
    return eps.real.copy(), -eps.imag


def debye(omega, eps_inf, d_eps, tau0):
    """Single-pole Debye, Eq. 3: eps_inf + (eps_s - eps_inf) / (1 + j w tau0)."""
    return eps_inf + d_eps / (1.0 + 1j * omega * tau0)


def havriliak_negami(omega, eps_inf, d_eps, tau0, alpha, beta):
    """Havriliak-Negami, Eq. 4: eps_inf + d_eps / (1 + (j w tau0)^alpha)^beta."""
    jwt = 1j * omega * tau0
    return eps_inf + d_eps / (1.0 + jwt ** alpha) ** beta


def cole_cole(omega, eps_inf, d_eps, tau0, alpha):
    """Cole-Cole: Eq. 4 with beta = 1 (Sec. II-B)."""
    return havriliak_negami(omega, eps_inf, d_eps, tau0, alpha, 1.0)


def cole_davidson(omega, eps_inf, d_eps, tau0, beta):
    """Cole-Davidson: Eq. 4 with alpha = 1 (Sec. II-B)."""
    return havriliak_negami(omega, eps_inf, d_eps, tau0, 1.0, beta)


def jonscher_eq5(omega, eps_inf, a_p, omega_p, n_p):
    """Jonscher as printed in Eq. 5: eps_inf + A_p (-j w / w_p)^n_p."""
    return eps_inf + a_p * (-1j * omega / omega_p) ** n_p


def jonscher(omega, eps_inf, a_p, omega_p, n_p):
    """Jonscher constant-Q form used by the benchmark workloads:
    eps_inf + a_p (w / w_p)^(n_p - 1) [1 - j cot(n_p pi / 2)].
    (Eq. 5 as printed, A_p(-j w/w_p)^n, has loss ratio tan(n pi/2) instead of
    cot(n pi/2); both are provided, see `jonscher_eq5`.)"""
    return eps_inf + a_p * (omega / omega_p) ** (n_p - 1.0) * (1.0 - 1j / math.tan(n_p * math.pi / 2))


def crim(omega, fractions, components, a=0.5):
    """CRIM, Eq. 6: eps^a = sum_i f_i eps_i^a, each component a Debye pole
    (eps_inf_i, d_eps_i, tau_i); a lossless constant has d_eps_i = 0."""
    acc = np.zeros(np.shape(omega), dtype=np.complex128)
    for f, (ei, de, tau) in zip(fractions, components):
        acc = acc + f * debye(omega, ei, de, tau) ** a
    return acc ** (1.0 / a)


def multi_debye(omega, eps_inf, d_eps, tau):
    """Multi-pole Debye expansion, Eq. 7: eps_inf + sum_n d_eps_n / (1 + j w tau_n)."""
    omega = np.asarray(omega, dtype=np.float64)
    d_eps = np.asarray(d_eps, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    return eps_inf + (d_eps[None, :] / (1.0 + 1j * omega[:, None] * tau[None, :])).sum(axis=1)


def synthesize(batch: W.Batch):
    """eps', eps'' of every spectrum of a workload batch, concatenated (CSR order).

    Model ids and parameter records are those documented in `workloads`.
    Debye-sum spectra get multiplicative noise eps' (1 + sigma z1), eps'' (1 + sigma z2).
    """
    re = np.zeros(batch.omega.shape[0])
    im = np.zeros(batch.omega.shape[0])
    for s in range(batch.S):
        a, b = batch.offsets[s], batch.offsets[s + 1]
        om = batch.omega[a:b]
        m, p = int(batch.model[s]), batch.params[s]
        if m == W.MODEL_DEBYE:
            eps = debye(om, p[0], p[1], p[2])
        elif m in (W.MODEL_HN, W.MODEL_CC, W.MODEL_CD):
            eps = havriliak_negami(om, p[0], p[1], p[2], p[3], p[4])
        elif m == W.MODEL_JONSCHER:
            eps = jonscher(om, p[0], p[1], p[2], p[3])
        elif m == W.MODEL_JONSCHER_EQ5:
            eps = jonscher_eq5(om, p[0], p[1], p[2], p[3])
        elif m == W.MODEL_CRIM:
            ncomp = int(p[1])
            fr = p[2:2 + ncomp]
            comps = [tuple(p[5 + 3 * i:8 + 3 * i]) for i in range(ncomp)]
            eps = crim(om, fr, comps, a=p[0])
        elif m == W.MODEL_DEBYE_SUM:
            pa, pb = batch.pole_offsets[s], batch.pole_offsets[s + 1]
            eps = multi_debye(om, p[0], batch.pole_deps[pa:pb], batch.pole_tau[pa:pb])
            eps = eps + jonscher(om, 0.0, p[1], p[2], p[3])
        else:
            raise ValueError(f"model id {m} has no synthesis")
        r, i = split(eps)
        if m == W.MODEL_DEBYE_SUM and batch.noise_re is not None:
            r = r * (1.0 + p[4] * batch.noise_re[a:b])
            i = i * (1.0 + p[4] * batch.noise_im[a:b])
        re[a:b] = r
        im[a:b] = i
    return re, im
