"""Whole fit of one spectrum and the reported result (oracle).

Sequence (Sec. III-B, IV): particle swarm (or differential evolution) over
log10(tau) with DLS weights per candidate (damping LAM_SEARCH), projected L-BFGS polish of the best `topk`
personal bests (lowest cost first, lowest particle index on ties), the best
polished candidate (lowest cost, lowest rank on ties) re-solved with damping
LAM_FINAL (by default the search damping: the reported weights are the DLS
weights of the found relaxation times) and the sign flip, poles sorted by
ascending tau. The result is the
record the paper emits (Listing 2): eps_inf, then (d_eps_n, tau_n).
"""
from __future__ import annotations

import numpy as np

from . import da, de, dls, lbfgs, pso, varpro


def fit_spectrum(omega, eps_re, eps_im, N: int, lo: float, hi: float, P: int, iters: int,
                 seed: int = 0, spectrum: int = 0, topk: int = 8, polish_iters: int = 50,
                 lam_search: float = dls.LAM_SEARCH, lam_final: float = dls.LAM_FINAL,
                 method: str = "pso", de_opts: dict | None = None):
    """method "pso" (particle swarm), "de" (differential evolution) or "da" (dual
    annealing); keyword arguments of de.de / da.da in de_opts; the polish starts
    from the best personal bests (swarm), population members (evolution) or chain
    states (annealing)."""
    def cost_fn(th):
        return dls.cost_population(omega, eps_re, eps_im, th, lam_search)[0]

    if method == "pso":
        pbx, pbc, gi, trace = pso.pso(cost_fn, N, lo, hi, P, iters, seed, spectrum)
    elif method == "de":
        pbx, pbc, gi, trace = de.de(cost_fn, N, lo, hi, P, iters, seed, spectrum, **(de_opts or {}))
    elif method == "da":
        pbx, pbc, gi, trace = da.da(cost_fn, N, lo, hi, P, iters, seed, spectrum, **(de_opts or {}))
    else:
        raise ValueError("method must be 'pso', 'de' or 'da'")
    order = np.argsort(pbc, kind="stable")
    best_th, best_c = pbx[gi].copy(), float(pbc[gi])
    n_evals = P * (iters * 2 * N + 1) if method == "da" else P * (iters + 1)
    polished = []
    for rank in range(min(topk, P)):
        th0 = pbx[order[rank]]
        th, c, ne = lbfgs.polish(lambda t: varpro.cost_grad(omega, eps_re, eps_im, t, lam_search),
                                 th0, lo, hi, polish_iters)
        n_evals += ne
        polished.append((c, rank, th))
    if polished:
        c, _, th = min(polished, key=lambda e: (e[0], e[1]))
        best_th, best_c = th, c
    cfin, w = dls.cost(omega, eps_re, eps_im, best_th[None, :], lam_final, return_weights=True)
    w = w[0]
    order_t = np.argsort(best_th, kind="stable")
    tau = 10.0 ** best_th[order_t]
    d_eps = w[1:][order_t]
    theta_sorted = best_th[order_t]
    return {
        "eps_inf": float(w[0]),
        "d_eps": d_eps,
        "tau": tau,
        "theta": theta_sorted,
        "cost_search": float(best_c),
        "cost_final": float(cfin[0]),
        "trace": trace,
        "n_evals": n_evals,
        "avg_frac_err": dls.avg_fractional_error(omega, eps_re, eps_im,
                                                 np.concatenate([[w[0]], d_eps]), theta_sorted),
    }


def fitted_eps(omega, result) -> np.ndarray:
    """Complex permittivity of a fit result (Eq. 7)."""
    return dls.model_eps(omega, np.concatenate([[result["eps_inf"]], result["d_eps"]]),
                         np.log10(result["tau"]))


AUTO_THRESHOLD = 5.0   # percent
AUTO_N_MAX = 20


def fit_auto(omega, eps_re, eps_im, lo: float, hi: float, P: int, iters: int, seed: int = 0,
             spectrum: int = 0, topk: int = 8, polish_iters: int = 50, n_hi: int = AUTO_N_MAX,
             threshold: float = AUTO_THRESHOLD, **kw):
    """Automatic number of poles (Sec. III-B, N = -1): fit with N = 1, 2, ... poles
    and stop at the first N whose average fractional error (Sec. IV metric, in
    percent: mean relative error of eps' plus that of eps'') is below `threshold`,
    or at N = n_hi (the paper's cap is 20 poles and 5 %). Every N is a complete
    fit of its own with the same seed and spectrum index. Returns that fit's
    record with "N" added."""
    for N in range(1, n_hi + 1):
        r = fit_spectrum(omega, eps_re, eps_im, N, lo, hi, P, iters, seed=seed, spectrum=spectrum,
                         topk=topk, polish_iters=polish_iters, **kw)
        if r["avg_frac_err"] < threshold:
            break
    r["N"] = N
    return r
