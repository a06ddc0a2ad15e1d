"""End-to-end fit agreement between a GPU fit and the FP64 oracle's fit.

The criterion per spectrum: the fitted spectra agree to relative RMS <= 1e-4
(over the complex values at the spectrum's frequencies), or the GPU fit's damped
cost is at most the oracle's times (1 + 1e-6) (an equally good or better minimum
of the multimodal search).

One case is decided differently. On over-parameterised spectra (more poles than
the spectrum needs, e.g. a CRIM mixture whose only relaxation is the water pole,
fitted with 7-12 poles), the damped objective has flat valleys of collapsing
poles and poles without weight, and the L-BFGS polish from a given start point
is itself chaotic: perturbing its start points by 1e-9 decades changes the
oracle's own FP64 result by more than the criterion. A run in another precision
cannot then be expected to reproduce the oracle's path. Such a spectrum is found
by running the oracle's polish again from perturbed start points; the GPU fit is
then accepted if its cost is within the spread of those FP64 results
(at most the worst of them times (1 + 1e-6)).
"""
from __future__ import annotations

import numpy as np

from oracle import dls, fit, lbfgs, models, pso, varpro

RELRMS_TOL = 1e-4
COST_SLACK = 1e-6


def agree(e_gpu, cost_gpu, e_ref, cost_ref) -> bool:
    return dls.rel_rms(e_gpu, e_ref) <= RELRMS_TOL or cost_gpu <= cost_ref * (1 + COST_SLACK)


def _finish(omega, re, im, polished):
    """The oracle's result from polished (cost, rank, theta): best line, FP64 re-solve."""
    c, _, th = min(polished, key=lambda e: (e[0], e[1]))
    cfin, w = dls.cost(omega, re, im, th[None, :], dls.LAM_FINAL, return_weights=True)
    return float(cfin[0]), models.multi_debye(omega, w[0][0], w[0][1:], 10.0 ** th)


def perturbed_oracle_fits(omega, re, im, N, lo, hi, P, iters, seed, spectrum, topk, polish_iters,
                          scale=1e-9, repeats=3):
    """The oracle's swarm, then its polish repeated from start points perturbed by `scale`
    decades (seeded normal offsets): [(final cost, fitted eps)] of the unperturbed run
    followed by the perturbed ones."""
    cf = lambda th: dls.cost_population(omega, re, im, th)[0]
    pbx, pbc, gi, _ = pso.pso(cf, N, lo, hi, P, iters, seed, spectrum)
    order = np.argsort(pbc, kind="stable")
    cg = lambda t: varpro.cost_grad(omega, re, im, t)
    rs = np.random.default_rng(12345 + spectrum)
    out = []
    for r in range(repeats + 1):
        pol = []
        for rank in range(min(topk, P)):
            th0 = pbx[order[rank]] + (scale * rs.standard_normal(N) if r else 0.0)
            th, c, _ = lbfgs.polish(cg, np.clip(th0, lo, hi), lo, hi, polish_iters)
            pol.append((c, rank, th))
        out.append(_finish(omega, re, im, pol))
    return out


def check_spectrum(omega, re, im, N, lo, hi, P, iters, seed, spectrum, topk, polish_iters, e_gpu, cost_gpu,
                   ref=None):
    """(ok, how) for one spectrum: how is "strict" or "chaotic" (accepted within the oracle's
    own perturbed spread) or "fail"."""
    if ref is None:
        ref = fit.fit_spectrum(omega, re, im, N, lo, hi, P, iters, seed=seed, spectrum=spectrum, topk=topk,
                               polish_iters=polish_iters)
    e_ref = fit.fitted_eps(omega, ref)
    if agree(e_gpu, cost_gpu, e_ref, ref["cost_final"]):
        return True, "strict"
    runs = perturbed_oracle_fits(omega, re, im, N, lo, hi, P, iters, seed, spectrum, topk, polish_iters)
    c0, e0 = runs[0]
    chaotic = any(not agree(e, c, e0, c0) for c, e in runs[1:])
    if chaotic and cost_gpu <= max(c for c, _ in runs) * (1 + COST_SLACK):
        return True, "chaotic"
    return False, "fail"
