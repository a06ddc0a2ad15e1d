"""Particle-swarm search over log10(tau) (oracle).

The paper's default optimiser is particle swarm optimisation (Kennedy and
Eberhart) over the relaxation times, with the weights of every particle found
by damped least squares (Sec. III-A, III-B); its implementation builds on the
pyswarm package. The paper states neither coefficients, stopping rule nor
update order. Readings taken here:
  * particle position theta in [lo, hi]^N (log10 tau), clamped to the bounds;
  * initial positions U[lo, hi], initial velocities U[-(hi-lo), hi-lo];
  * inertia omega = 0.5, cognitive phi_p = 0.5, social phi_g = 0.5 (pyswarm's
    documented defaults), fresh r1, r2 ~ U[0,1) per particle and dimension;
  * synchronous update: the whole population is evaluated, then personal bests
    (replaced only on a strictly lower cost) and the global best (lowest cost,
    lowest particle index on ties) are updated;
  * a fixed number of generations, no early stop; non-finite costs count as +inf.
Random numbers come from `rng` keyed by (seed, tag, spectrum, generation,
particle, dim).
"""
from __future__ import annotations

import numpy as np

from . import rng

OMEGA = 0.5
PHI_P = 0.5
PHI_G = 0.5


def _finite(c):
    c = np.asarray(c, dtype=np.float64)
    return np.where(np.isfinite(c), c, np.inf)


def pso(cost_fn, N: int, lo: float, hi: float, P: int, iters: int, seed: int = 0,
        spectrum: int = 0, omega: float = OMEGA, phi_p: float = PHI_P, phi_g: float = PHI_G):
    """Run the swarm. cost_fn maps thetas (P, N) to costs (P,).

    Returns (pbest_theta (P,N), pbest_cost (P,), gbest index, trace of the global
    best cost after each evaluation round (iters+1,)).
    """
    span = hi - lo
    x = lo + span * rng.uniform_array(seed, rng.TAG_INIT_POS, spectrum, 0, P, N)
    v = -span + 2.0 * span * rng.uniform_array(seed, rng.TAG_INIT_VEL, spectrum, 0, P, N)
    c = _finite(cost_fn(x))
    pbx, pbc = x.copy(), c.copy()
    gi = int(np.argmin(pbc))
    trace = [pbc[gi]]
    for g in range(1, iters + 1):
        r1 = rng.uniform_array(seed, rng.TAG_R1, spectrum, g, P, N)
        r2 = rng.uniform_array(seed, rng.TAG_R2, spectrum, g, P, N)
        v = omega * v + phi_p * r1 * (pbx - x) + phi_g * r2 * (pbx[gi][None, :] - x)
        x = np.clip(x + v, lo, hi)
        c = _finite(cost_fn(x))
        better = c < pbc
        pbx[better] = x[better]
        pbc[better] = c[better]
        gi = int(np.argmin(pbc))
        trace.append(pbc[gi])
    return pbx, pbc, gi, np.array(trace)
