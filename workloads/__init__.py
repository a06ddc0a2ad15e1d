"""Seeded synthetic workloads for multi-Debye fitting.

This module only DRAWS inputs: which relaxation model each spectrum follows,
its parameters, the frequency grid, the pole count N, the log10(tau) search
bounds, fed-in candidate populations and measurement noise. It evaluates none
of the fitting method's arithmetic: turning the drawn parameters into
permittivity values (Eqs. 4-7) is done separately by the oracle (numpy, FP64)
and by the CUDA library (its target-synthesis kernel).

Both the oracle and the CUDA path consume what this module returns, so both
see bit-identical inputs.

Workload shapes follow the paper's own example (Sec. IV: Havriliak-Negami,
10 MHz-100 GHz, N=5) and these named workloads:

  single_hn_k50          one HN target, K=50, N=3, P=64, 100 iterations
  mixed_1024             1024 spectra, models drawn from HN / Cole-Cole /
                         Cole-Davidson / Jonscher / CRIM, K in [50,1000],
                         N in [2,12], P=256, 200 iterations (solved in FP64 or
                         in mixed precision: same inputs)
  hn_256_k2000           256 HN spectra, K=2000, N=8, 4096 fed-in candidates
                         per spectrum
  tabulated_16384_k4096  16384 tabulated spectra (40-pole Debye sum + Jonscher
                         tail + 1 % multiplicative Gaussian noise), K=4096,
                         N=20, P=512, 100 generations

Model ids (shared vocabulary of the library's C ABI):
  0 Debye, 1 Havriliak-Negami, 2 Cole-Cole, 3 Cole-Davidson,
  4 Jonscher (constant-Q form eps_inf + a_p (w/w_p)^(n-1) [1 - j cot(n pi/2)]),
  5 Jonscher as printed in Eq. 5 (eps_inf + A_p (-j w/w_p)^n),
  6 CRIM (Eq. 6) of up to three Debye components,
  7 Debye sum + Jonscher tail (the synthetic "tabulated" spectra),
  8 tabulated (values supplied directly).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MODEL_DEBYE = 0
MODEL_HN = 1
MODEL_CC = 2
MODEL_CD = 3
MODEL_JONSCHER = 4
MODEL_JONSCHER_EQ5 = 5
MODEL_CRIM = 6
MODEL_DEBYE_SUM = 7
MODEL_TABULATED = 8

N_PARAMS = 16  # fixed-size per-spectrum parameter record (see param layout below)

# Parameter record layout (float64[N_PARAMS]) per model id:
#   Debye/HN/CC/CD : [eps_inf, d_eps, tau0, alpha, beta]
#   Jonscher (4,5) : [eps_inf, a_p, omega_p, n_p]
#   CRIM           : [a, m, f_1, f_2, f_3, einf_1, deps_1, tau_1, einf_2, deps_2,
#                     tau_2, einf_3, deps_3, tau_3]   (m <= 3 components)
#   Debye sum      : [eps_inf, a_p, omega_p, n_p, noise_sigma]; the poles live
#                    in the ragged pole arrays, the noise in noise_re/noise_im

# CRIM components of the 1024-spectrum workload: free water as a Debye pole,
# sand and air as lossless constants.
WATER = (4.9, 75.0, 9.23e-12)
SAND = (4.5, 0.0, 1.0)
AIR = (1.0, 0.0, 1.0)

OMEGA_P = 2.0 * math.pi * 1e8


@dataclass
class Batch:
    """A ragged batch of S spectra (CSR over frequencies)."""
    name: str
    offsets: np.ndarray          # int64[S+1]
    omega: np.ndarray            # float64[sum K], rad/s, log-spaced per spectrum
    model: np.ndarray            # int32[S]
    params: np.ndarray           # float64[S, N_PARAMS]
    n_poles: np.ndarray          # int32[S]   fitted Debye poles N
    lo: np.ndarray               # float64[S] log10(tau) lower bound
    hi: np.ndarray               # float64[S] log10(tau) upper bound
    pole_offsets: np.ndarray     # int64[S+1] (model 7 only, else all zero)
    pole_tau: np.ndarray         # float64[total poles]
    pole_deps: np.ndarray        # float64[total poles]
    noise_re: np.ndarray | None  # float64[sum K] standard normals or None
    noise_im: np.ndarray | None
    P: int = 64                  # population size
    iters: int = 100             # PSO generations after initialisation
    extra: dict = field(default_factory=dict)

    @property
    def S(self) -> int:
        return int(self.model.shape[0])

    @property
    def K(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def n_max(self) -> int:
        return int(self.n_poles.max()) if self.S else 0

    def subset(self, idx) -> "Batch":
        """Spectra idx (in order) as a new, self-contained batch."""
        idx = np.asarray(idx, dtype=np.int64)
        K = self.K[idx]
        offs = np.concatenate([[0], np.cumsum(K)]).astype(np.int64)
        om = np.concatenate([self.omega[self.offsets[s]:self.offsets[s + 1]] for s in idx]) \
            if len(idx) else np.zeros(0)
        def cat(a):
            if a is None:
                return None
            return np.concatenate([a[self.offsets[s]:self.offsets[s + 1]] for s in idx]) \
                if len(idx) else np.zeros(0)
        npol = np.diff(self.pole_offsets)[idx]
        poffs = np.concatenate([[0], np.cumsum(npol)]).astype(np.int64)
        ptau = np.concatenate([self.pole_tau[self.pole_offsets[s]:self.pole_offsets[s + 1]]
                               for s in idx]) if len(idx) else np.zeros(0)
        pdeps = np.concatenate([self.pole_deps[self.pole_offsets[s]:self.pole_offsets[s + 1]]
                                for s in idx]) if len(idx) else np.zeros(0)
        return Batch(self.name + f"[{len(idx)}]", offs, om, self.model[idx].copy(),
                     self.params[idx].copy(), self.n_poles[idx].copy(), self.lo[idx].copy(),
                     self.hi[idx].copy(), poffs, ptau, pdeps, cat(self.noise_re),
                     cat(self.noise_im), self.P, self.iters, dict(self.extra))


def log_grid(f_lo: float, f_hi: float, K: int) -> np.ndarray:
    """Angular frequencies 2*pi*f, f log-spaced with both endpoints included."""
    return 2.0 * math.pi * np.logspace(math.log10(f_lo), math.log10(f_hi), K)


def _assemble(name, Ks, f_lo, f_hi, model, params, n_poles, lo, hi, P, iters,
              poles=None, noise=None, extra=None) -> Batch:
    S = len(Ks)
    offs = np.concatenate([[0], np.cumsum(Ks)]).astype(np.int64)
    omega = np.concatenate([log_grid(f_lo, f_hi, int(k)) for k in Ks]) if S else np.zeros(0)
    if poles is None:
        poffs = np.zeros(S + 1, dtype=np.int64)
        ptau = np.zeros(0)
        pdeps = np.zeros(0)
    else:
        ptau, pdeps, npol = poles
        poffs = np.concatenate([[0], np.cumsum(npol)]).astype(np.int64)
    nre, nim = (None, None) if noise is None else noise
    return Batch(name, offs, omega, np.asarray(model, np.int32), np.asarray(params, np.float64),
                 np.asarray(n_poles, np.int32), np.asarray(lo, np.float64),
                 np.asarray(hi, np.float64), poffs, np.asarray(ptau, np.float64),
                 np.asarray(pdeps, np.float64), nre, nim, P, iters, extra or {})


def _rng(seed: int, tag: str) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, sum(ord(c) << (8 * i) for i, c in enumerate(tag))]))


def single_hn(eps_inf=3.4, d_eps=2.7, tau0=8e-10, alpha=0.91, beta=0.45, f_lo=1e8, f_hi=1e10,
              K=50, N=3, lo=-13.0, hi=-6.0, P=64, iters=100, name="single_hn_k50") -> Batch:
    """One Havriliak-Negami spectrum (defaults: the 50-point single-target workload)."""
    p = np.zeros((1, N_PARAMS))
    p[0, :5] = [eps_inf, d_eps, tau0, alpha, beta]
    return _assemble(name, [K], f_lo, f_hi, [MODEL_HN], p, [N], [lo], [hi], P, iters)


def paper_example(K=200, N=5, P=64, iters=100) -> Batch:
    """The paper's worked example (Sec. IV, Listing 1): HN with eps_inf=2.7,
    eps_s-eps_inf=5.9, tau0=0.94 ns (9.4e-10 s), alpha=0.91, beta=0.45,
    10 MHz-100 GHz, N=5 poles. K is not stated in the paper."""
    return single_hn(2.7, 5.9, 9.4e-10, 0.91, 0.45, 1e7, 1e11, K, N, -13.0, -6.0, P, iters,
                     name="paper_example")


def _draw_model_params(rng, model: int) -> np.ndarray:
    p = np.zeros(N_PARAMS)
    eps_inf = rng.uniform(2.0, 8.0)
    if model in (MODEL_HN, MODEL_CC, MODEL_CD):
        d_eps = rng.uniform(1.0, 80.0)
        tau0 = 10.0 ** rng.uniform(-11.0, -8.0)
        alpha = rng.uniform(0.3, 1.0)
        beta = rng.uniform(0.3, 1.0)
        if model == MODEL_CC:
            beta = 1.0
        if model == MODEL_CD:
            alpha = 1.0
        p[:5] = [eps_inf, d_eps, tau0, alpha, beta]
    elif model in (MODEL_JONSCHER, MODEL_JONSCHER_EQ5):
        n_p = rng.uniform(0.3, 0.9)
        a_p = rng.uniform(1.0, 10.0)
        p[:4] = [eps_inf, a_p, OMEGA_P, n_p]
    elif model == MODEL_CRIM:
        f = rng.dirichlet([1.0, 1.0, 1.0])
        p[:2] = [0.5, 3]
        p[2:5] = f
        p[5:8] = WATER
        p[8:11] = SAND
        p[11:14] = AIR
    else:
        raise ValueError(model)
    return p


def mixed_batch(S=1024, seed=0, P=256, iters=200, K_range=(50, 1000), N_range=(2, 12),
                f_lo=1e6, f_hi=1e10, lo=-13.0, hi=-5.0, name="mixed_1024") -> Batch:
    """Ragged batch of HN / CC / CD / Jonscher / CRIM spectra (the 1024-spectrum
    workload): eps_inf U[2,8], d_eps U[1,80], log10 tau0 U[-11,-8], alpha,beta U[0.3,1],
    n U[0.3,0.9], a_p U[1,10], w_p = 2 pi 1e8, CRIM fractions Dirichlet(1,1,1);
    K uniform in K_range, N uniform in N_range."""
    rng = _rng(seed, "DATA/mixed")
    models = rng.choice([MODEL_HN, MODEL_CC, MODEL_CD, MODEL_JONSCHER, MODEL_CRIM], size=S)
    params = np.stack([_draw_model_params(rng, int(m)) for m in models]) if S else \
        np.zeros((0, N_PARAMS))
    Ks = rng.integers(K_range[0], K_range[1] + 1, size=S)
    Ns = rng.integers(N_range[0], N_range[1] + 1, size=S)
    return _assemble(name, Ks, f_lo, f_hi, models, params, Ns, np.full(S, lo), np.full(S, hi),
                     P, iters)


def hn_batch(S=256, seed=0, K=2000, N=8, P=4096, f_lo=1e6, f_hi=1e10, lo=-13.0, hi=-5.0,
             name="hn_256_k2000") -> Batch:
    """S Havriliak-Negami spectra with the 1024-spectrum workload's parameter ranges,
    fixed K and N (the differentiation workload)."""
    rng = _rng(seed, "DATA/hn")
    params = np.stack([_draw_model_params(rng, MODEL_HN) for _ in range(S)])
    return _assemble(name, np.full(S, K), f_lo, f_hi, np.full(S, MODEL_HN), params,
                     np.full(S, N), np.full(S, lo), np.full(S, hi), P, 50)


def tabulated_batch(S=16384, seed=0, K=4096, N=20, P=512, iters=100, n_src_poles=40,
                    f_lo=1e5, f_hi=1e10, lo=-13.0, hi=-5.0, noise_sigma=0.01,
                    name="tabulated_16384_k4096") -> Batch:
    """Synthetic 'measured' spectra: a sum of 40 Debye poles (log10 tau U[-12,-6],
    d_eps log-uniform [0.1,20], eps_inf U[2,8]) plus a Jonscher tail (a_p U[1,10],
    n U[0.3,0.9], w_p = 2 pi 1e8, no extra eps_inf) with 1 % multiplicative Gaussian
    noise on eps' and eps''."""
    rng = _rng(seed, "DATA/tab")
    params = np.zeros((S, N_PARAMS))
    params[:, 0] = rng.uniform(2.0, 8.0, S)
    params[:, 1] = rng.uniform(1.0, 10.0, S)
    params[:, 2] = OMEGA_P
    params[:, 3] = rng.uniform(0.3, 0.9, S)
    params[:, 4] = noise_sigma
    ptau = 10.0 ** rng.uniform(-12.0, -6.0, S * n_src_poles)
    pdeps = 10.0 ** rng.uniform(math.log10(0.1), math.log10(20.0), S * n_src_poles)
    z = rng.standard_normal((2, S * K))
    return _assemble(name, np.full(S, K), f_lo, f_hi, np.full(S, MODEL_DEBYE_SUM), params,
                     np.full(S, N), np.full(S, lo), np.full(S, hi), P, iters,
                     poles=(ptau, pdeps, np.full(S, n_src_poles)), noise=(z[0], z[1]))


WORKLOADS = ("single_hn_k50", "mixed_1024", "hn_256_k2000", "tabulated_16384_k4096")


def workload(name: str, seed: int = 0) -> Batch:
    """A named workload (see the module docstring)."""
    if name == "single_hn_k50":
        return single_hn()
    if name == "mixed_1024":
        return mixed_batch(seed=seed)
    if name == "hn_256_k2000":
        return hn_batch(seed=seed)
    if name == "tabulated_16384_k4096":
        return tabulated_batch(seed=seed)
    raise KeyError(name)


def population(batch: Batch, P: int, seed: int = 0, tag: str = "POP") -> np.ndarray:
    """Fed-in candidate populations theta[S, P, n_max] = log10(tau), uniform within each
    spectrum's bounds; entries beyond a spectrum's N are zero (ignored)."""
    rng = _rng(seed, tag)
    S, nmax = batch.S, batch.n_max
    u = rng.uniform(0.0, 1.0, size=(S, P, nmax))
    th = batch.lo[:, None, None] + (batch.hi - batch.lo)[:, None, None] * u
    mask = np.arange(nmax)[None, None, :] < batch.n_poles[:, None, None]
    return np.where(mask, th, 0.0)
