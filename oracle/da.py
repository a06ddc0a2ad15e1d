"""Dual annealing over log10(tau) (oracle).

The paper lists dual annealing (generalized simulated annealing, Tsallis and
Stariolo, Physica A 233, 1996; the "dual" variant of Xiang et al., 1997, adds
a local search) among its optimisers for the relaxation times (Sec. III-B),
built on SciPy optimize, with the weights of every candidate from damped least
squares. It states no schedule or parameters. Readings taken here:
  * P independent chains per spectrum, started at U[lo, hi]^N (the swarm's
    initial positions); the local search is the common L-BFGS polish of the
    best chain states after the annealing;
  * visiting parameter qv = 2.62, acceptance parameter qa = -5, initial
    temperature T0 = 5230 (SciPy's documented defaults);
  * outer iteration t = 1, 2, ...: visiting temperature
        T(t) = T0 (2^(qv-1) - 1) / ((1 + t)^(qv-1) - 1),
    acceptance temperature T(t) / t;
  * each outer iteration is a Markov chain of 2N moves: moves j < N displace
    every coordinate, moves j >= N only coordinate j - N;
  * a displacement is a deviate of the Tsallis visiting distribution,
        dx = sigma(T) z1 / |z2|^((qv-1)/(3-qv)),  z1, z2 ~ N(0, 1),
        sigma(T) = exp((log T - C) / (3 - qv)),
    the ratio method of Mantegna (Phys. Rev. E 49, 1994) with the scale of
    the distribution of width T^(1/(3-qv)); C = (qv-1) log(A / B) with
        A = pi (1-a) / sin(pi (1-a)) / Gamma(2 - a),  a = 1/(qv-1) - 1/2,
        B = sqrt(pi) (qv-1)^(4-qv) / (2^((2-qv)/(qv-1)) (3-qv)),
    evaluated once to 40 digits (C_QV below); |dx| is capped at 1e8;
  * a coordinate leaving [lo, hi] is wrapped back periodically:
        lo + ((x - lo) mod (hi - lo));
  * generalized Metropolis acceptance: a lower energy is always accepted;
    otherwise with probability [1 - (1-qa) dE / T_acc]^(1/(1-qa)) (zero if
    the bracket is not positive), compared with a uniform draw u <= p;
  * each chain keeps its best state (strictly lower cost replaces); the trace
    is the lowest best cost of all chains after each outer iteration; at most
    1000 outer iterations, so the temperature never falls to the re-annealing
    threshold (2e-5 T0) and chains are not restarted;
  * non-finite costs count as +inf (never accepted).
log and exp are the fixed-operation versions of `dmath`; the Gaussian pairs use
the polar method with up to 32 tries, try k of coordinate d in move j drawing
the uniforms at slot ((j * 20 + d) * 32 + k) * 2 + {0, 1}. Random numbers
come from `rng` keyed by (seed, tag, spectrum, outer iteration, chain, slot).
"""
from __future__ import annotations

import numpy as np

from . import dmath, rng

T0 = 5230.0
QV = 2.62
QA = -5.0
C_QV = -0.6233798028078907   # (qv-1) log(A/B) at qv = 2.62, from a 40-digit evaluation
TAIL = 1.0e8
MAX_ITERS = 1000
NMAX = 20


def _finite(c):
    c = np.asarray(c, dtype=np.float64)
    return np.where(np.isfinite(c), c, np.inf)


def visiting_temperature(t: int, t0: float = T0) -> float:
    """T(t) of outer iteration t >= 1."""
    num = dmath.exp((QV - 1.0) * dmath.log(2.0)) - 1.0
    den = dmath.exp((QV - 1.0) * dmath.log(float(t) + 1.0)) - 1.0
    return (t0 * num) / den


def sigma(T: float) -> float:
    return dmath.exp((dmath.log(T) - C_QV) / (3.0 - QV))


def _slot(j: int, d: int, k: int, which: int) -> int:
    return ((j * NMAX + d) * dmath.POLAR_TRIES + k) * 2 + which


def gauss_pairs(seed: int, spectrum: int, t: int, P: int, j: int, dims) -> tuple[np.ndarray, np.ndarray]:
    """Polar-method normal pairs (z1, z2) of move j for coordinates `dims`, all chains: (P, len(dims))."""
    us, vs = [], []
    for k in range(dmath.POLAR_TRIES):
        us.append(rng.uniform_cols(seed, rng.TAG_DA_VISIT, spectrum, t, P, [_slot(j, d, k, 0) for d in dims]))
        vs.append(rng.uniform_cols(seed, rng.TAG_DA_VISIT, spectrum, t, P, [_slot(j, d, k, 1) for d in dims]))
    return dmath.gauss_pair(us, vs)


def visit(z1, z2, sig: float):
    """Visiting deviates from normal pairs; |z2| = 0 gives the capped tail."""
    az = np.abs(z2)
    den = dmath.exp(((QV - 1.0) / (3.0 - QV)) * dmath.log(np.where(az > 0.0, az, 1.0)))
    dx = np.where(az > 0.0, (sig * z1) / den, np.copysign(TAIL, z1))
    return np.clip(dx, -TAIL, TAIL)


def wrap(x, lo: float, hi: float):
    span = hi - lo
    r = np.fmod(x - lo, span)
    r = np.where(r < 0.0, r + span, r)
    return np.where((x < lo) | (x > hi), lo + r, x)


def accept_probability(de, t_acc: float, qa: float = QA):
    """Generalized Metropolis probability of an uphill move de > 0."""
    tmp = 1.0 - ((1.0 - qa) * de) / t_acc
    pos = tmp > 0.0
    return np.where(pos, dmath.exp(dmath.log(np.where(pos, tmp, 1.0)) / (1.0 - qa)), 0.0)


def da(cost_fn, N: int, lo: float, hi: float, P: int, iters: int, seed: int = 0, spectrum: int = 0,
       t0: float = T0, qa: float = QA):
    """Run the chains. cost_fn maps thetas (P, N) to costs (P,).

    Returns (best states (P,N), best costs (P,), index of the lowest, trace of the
    lowest best cost after each outer iteration (iters+1,)), the swarm's record."""
    if iters > MAX_ITERS:
        raise ValueError(f"at most {MAX_ITERS} outer iterations")
    x = lo + (hi - lo) * rng.uniform_array(seed, rng.TAG_INIT_POS, spectrum, 0, P, N)
    e = _finite(cost_fn(x))
    xb, eb = x.copy(), e.copy()
    trace = [float(np.min(eb))]
    for t in range(1, iters + 1):
        T = visiting_temperature(t, t0)
        sig = sigma(T)
        t_acc = T / float(t)
        for j in range(2 * N):
            dims = list(range(N)) if j < N else [j - N]
            z1, z2 = gauss_pairs(seed, spectrum, t, P, j, dims)
            xt = x.copy()
            xt[:, dims] = wrap(x[:, dims] + visit(z1, z2, sig), lo, hi)
            et = _finite(cost_fn(xt))
            u = rng.uniform_cols(seed, rng.TAG_DA_ACCEPT, spectrum, t, P, [j])[:, 0]
            down = et < e
            up_ok = np.isfinite(et) & ~down & (u <= accept_probability(et - e, t_acc, qa))
            acc = down | up_ok
            x[acc] = xt[acc]
            e[acc] = et[acc]
            better = e < eb
            xb[better] = x[better]
            eb[better] = e[better]
        trace.append(float(np.min(eb)))
    return xb, eb, int(np.argmin(eb)), np.array(trace)
