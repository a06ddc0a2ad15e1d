"""Differential evolution over log10(tau) (oracle).

The paper lists differential evolution (Storn and Price, J. Global Optim. 11,
1997) among its three optimisers for the relaxation times (Sec. III-B), with
the weights of every candidate from damped least squares as for the swarm, and
says that its optimisers build on SciPy's optimize module. It states no
strategy, coefficients or stopping rule. Readings taken here:
  * population theta in [lo, hi]^N (log10 tau), initial members U[lo, hi]
    (the swarm's initial positions: same generator keys);
  * mutation DE/rand/1 (Storn and Price's scheme): v = x_r1 + F (x_r2 - x_r3),
    or DE/best/1: v = x_best + F (x_r1 - x_r2), with r1, r2, r3 distinct and
    different from the target;
  * scale factor F drawn once per generation from U[f_lo, f_hi) (dither;
    SciPy's documented default range [0.5, 1)), crossover rate CR = 0.7
    (SciPy's documented default);
  * binomial crossover: coordinate d comes from the mutant when its uniform
    draw is below CR or d is the one coordinate j_rand drawn per member, else
    from the target;
  * a mutant coordinate outside [lo, hi] is replaced by a uniform draw in
    [lo, hi] (as SciPy does);
  * synchronous generations: every trial is evaluated, then a trial replaces
    its target only on a strictly lower cost (Storn and Price's selection);
    the best member is the lowest cost, lowest index on ties; non-finite costs
    count as +inf; a fixed number of generations, no early stop.
Random numbers come from `rng` keyed by (seed, tag, spectrum, generation,
member, slot).
"""
from __future__ import annotations

import numpy as np

from . import rng

F_LO = 0.5
F_HI = 1.0
CR = 0.7
RAND1 = 0
BEST1 = 1


def _finite(c):
    c = np.asarray(c, dtype=np.float64)
    return np.where(np.isfinite(c), c, np.inf)


def donors(seed: int, spectrum: int, generation: int, P: int, k: int) -> np.ndarray:
    """For every target p < P, k distinct member indices, all different from p, as (P, k).
    Slot j draws an integer r below P - 1 - j and takes the r-th smallest index (from 0)
    among those not yet taken (the target and slots 0..j-1)."""
    if P < k + 1:
        raise ValueError(f"differential evolution with {k} donors needs P >= {k + 1}")
    z = rng.key_array(seed, rng.TAG_DE_IDX, spectrum, generation, P, k)
    taken = np.arange(P, dtype=np.int64)[:, None]
    out = np.empty((P, k), dtype=np.int64)
    for j in range(k):
        r = ((z[:, j] >> np.uint64(32)) * np.uint64(P - 1 - j)) >> np.uint64(32)
        r = r.astype(np.int64)
        for e in np.sort(taken, axis=1).T:  # skip the taken indices in ascending order
            r = r + (r >= e)
        out[:, j] = r
        taken = np.concatenate([taken, r[:, None]], axis=1)
    return out


def trials(x, best: int, seed: int, spectrum: int, generation: int, lo: float, hi: float,
           f_lo: float = F_LO, f_hi: float = F_HI, cr: float = CR, strategy: int = RAND1):
    """Trial vectors (mutation + binomial crossover) of generation `generation` >= 1
    from the population x (P, N) whose best member is `best`."""
    P, N = x.shape
    span = hi - lo
    F = f_lo + (f_hi - f_lo) * rng.uniform(seed, rng.TAG_DE_F, spectrum, generation, 0, 0)
    if strategy == RAND1:
        r = donors(seed, spectrum, generation, P, 3)
        v = x[r[:, 0]] + F * (x[r[:, 1]] - x[r[:, 2]])
    elif strategy == BEST1:
        r = donors(seed, spectrum, generation, P, 2)
        v = x[best][None, :] + F * (x[r[:, 0]] - x[r[:, 1]])
    else:
        raise ValueError("strategy must be RAND1 or BEST1")
    out_of_box = (v < lo) | (v > hi)
    v = np.where(out_of_box, lo + span * rng.uniform_array(seed, rng.TAG_DE_BOUND, spectrum, generation, P, N), v)
    zj = rng.key_array(seed, rng.TAG_DE_J, spectrum, generation, P, 1)[:, 0]
    jr = (((zj >> np.uint64(32)) * np.uint64(N)) >> np.uint64(32)).astype(np.int64)
    take = (rng.uniform_array(seed, rng.TAG_DE_CR, spectrum, generation, P, N) < cr) | \
        (np.arange(N)[None, :] == jr[:, None])
    return np.where(take, v, x)


def de(cost_fn, N: int, lo: float, hi: float, P: int, iters: int, seed: int = 0, spectrum: int = 0,
       f_lo: float = F_LO, f_hi: float = F_HI, cr: float = CR, strategy: int = RAND1):
    """Run differential evolution. cost_fn maps thetas (P, N) to costs (P,).

    Returns (population (P,N), costs (P,), best index, trace of the best cost after
    each evaluation round (iters+1,)), the same record as the swarm's."""
    x = lo + (hi - lo) * rng.uniform_array(seed, rng.TAG_INIT_POS, spectrum, 0, P, N)
    c = _finite(cost_fn(x))
    gi = int(np.argmin(c))
    trace = [c[gi]]
    for g in range(1, iters + 1):
        u = trials(x, gi, seed, spectrum, g, lo, hi, f_lo, f_hi, cr, strategy)
        cu = _finite(cost_fn(u))
        better = cu < c
        x[better] = u[better]
        c[better] = cu[better]
        gi = int(np.argmin(c))
        trace.append(c[gi])
    return x, c, gi, np.array(trace)
