// Search kernels of libdebyefit: particle swarm and differential evolution
// (Sec. III-B), top-k selection, projected L-BFGS polish, final re-solve and
// result assembly.
//
// Swarm update order matches the reference arithmetic exactly: explicit
// __d*_rn operations (no FMA contraction) so that positions are bit-identical
// to an FP64 implementation evaluating
//   v = (omega v + (phi_p r1) (p - x)) + (phi_g r2) (g - x),  x = clip(x + v, lo, hi).
#include <cmath>

#include "dmath.cuh"
#include "launch.h"
#include "search.h"

namespace debyefit {

// Spectrum field of the generator's key: the caller's index map, else the batch index.
__device__ __forceinline__ uint64_t key_id(const SwarmArgs& a, int64_t s) {
  return a.rng_id ? (uint64_t)a.rng_id[s] : (uint64_t)s;
}

__global__ void k_pso_init(SwarmArgs a) {
  const int64_t Q = (int64_t)a.S * a.P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / a.P, p = q % a.P;
    const int N = a.n_poles[s];
    const double lo = a.lo[s], hi = a.hi[s], span = __dsub_rn(hi, lo);
    const uint64_t pp = rng_prefix(a.seed, TAG_INIT_POS, key_id(a, s), 0);
    const uint64_t pv = rng_prefix(a.seed, TAG_INIT_VEL, key_id(a, s), 0);
    for (int d = 0; d < a.nmax; ++d) {
      double x = 0.0, v = 0.0;
      if (d < N) {
        x = __dadd_rn(lo, __dmul_rn(span, rng_uniform(pp, p, d)));
        v = __dadd_rn(-span, __dmul_rn(__dmul_rn(2.0, span), rng_uniform(pv, p, d)));
      }
      a.x[q * a.nmax + d] = x;
      a.v[q * a.nmax + d] = v;
    }
  }
}

// A draw's 53-bit integer u (the uniform is u 2^-53) as a double, built from its
// IEEE-754 fields with integer operations (exact for u < 2^53): on GB300 an FP64
// conversion costs as much as any other FP64 operation.
__device__ __forceinline__ double u53_double(uint64_t u) {
  if (u == 0) return 0.0;
  const int e = 63 - __clzll((long long)u);   // position of the top bit, 0..52
  const uint64_t mant = (u << (52 - e)) & 0x000FFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | mant));
}

__global__ void k_pso_move(SwarmArgs a) {
  const int64_t Q = (int64_t)a.S * a.P;
  const int gen = *a.gen;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / a.P, p = q % a.P;
    const int N = a.n_poles[s];
    const double lo = a.lo[s], hi = a.hi[s];
    const int64_t gq = s * a.P + a.gbest[s];
    const uint64_t p1 = rng_prefix(a.seed, TAG_R1, key_id(a, s), (uint64_t)gen);
    const uint64_t p2 = rng_prefix(a.seed, TAG_R2, key_id(a, s), (uint64_t)gen);
    // phi r = phi (u 2^-53) = (phi 2^-53) u: the scaling by 2^-53 is exact, so both round
    // the same exact product once and the update stays bit-identical to phi * r (for any
    // |phi| >= 2^-969, where phi 2^-53 is still a normal number)
    const double cp = __dmul_rn(a.phi_p, 0x1p-53), cg = __dmul_rn(a.phi_g, 0x1p-53);
    for (int d = 0; d < N; ++d) {
      const double x = a.x[q * a.nmax + d], v = a.v[q * a.nmax + d];
      const double pb = a.pbx[q * a.nmax + d], gb = a.pbx[gq * a.nmax + d];
      const double u1 = u53_double(rng_key(p1, p, d) >> 11), u2 = u53_double(rng_key(p2, p, d) >> 11);
      const double t1 = __dmul_rn(a.omega, v);
      const double t2 = __dmul_rn(__dmul_rn(cp, u1), __dsub_rn(pb, x));
      const double t3 = __dmul_rn(__dmul_rn(cg, u2), __dsub_rn(gb, x));
      const double vn = __dadd_rn(__dadd_rn(t1, t2), t3);
      a.v[q * a.nmax + d] = vn;
      a.x[q * a.nmax + d] = fmin(fmax(__dadd_rn(x, vn), lo), hi);
    }
  }
}

// Differential evolution (Storn and Price): one trial vector per population member.
// The population lives in pbx/pbc (k_pso_best's strictly-lower replacement is
// the evolution's selection), the trials are written to x for evaluation.
//   donors: slot j draws r below P-1-j and takes the r-th free index (ascending),
//           free = not the target and not an earlier slot;
//   mutant: rand/1  x_r0 + F (x_r1 - x_r2)   best/1  x_best + F (x_r0 - x_r1),
//           F = f_lo + (f_hi - f_lo) u once per generation;
//   a mutant coordinate outside [lo, hi] is re-drawn uniformly in the box;
//   binomial crossover: coordinate d from the mutant if u_d < CR or d = j_rand.
// Explicit __d*_rn operations keep the trials bit-identical to an FP64
// implementation evaluating the same expressions.
__global__ void k_de_trial(SwarmArgs a) {
  const int64_t Q = (int64_t)a.S * a.P;
  const int gen = *a.gen;
  const int k = a.de_strategy == DEBYE_DE_RAND1 ? 3 : 2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / a.P;
    const int p = (int)(q % a.P);
    const int N = a.n_poles[s];
    const double lo = a.lo[s], hi = a.hi[s], span = __dsub_rn(hi, lo);
    const uint64_t pidx = rng_prefix(a.seed, TAG_DE_IDX, key_id(a, s), (uint64_t)gen);
    const uint64_t pj = rng_prefix(a.seed, TAG_DE_J, key_id(a, s), (uint64_t)gen);
    const uint64_t pcr = rng_prefix(a.seed, TAG_DE_CR, key_id(a, s), (uint64_t)gen);
    const uint64_t pb = rng_prefix(a.seed, TAG_DE_BOUND, key_id(a, s), (uint64_t)gen);
    const double uf = rng_uniform(rng_prefix(a.seed, TAG_DE_F, key_id(a, s), (uint64_t)gen), 0, 0);
    const double F = __dadd_rn(a.de_f_lo, __dmul_rn(__dsub_rn(a.de_f_hi, a.de_f_lo), uf));
    int taken[4];  // sorted ascending
    int r[3] = {0, 0, 0};
    taken[0] = p;
    int nt = 1;
    for (int j = 0; j < k; ++j) {
      int v = (int)rng_below(rng_key(pidx, (uint64_t)p, (uint64_t)j), (uint32_t)(a.P - 1 - j));
      for (int t = 0; t < nt; ++t) v += (v >= taken[t]) ? 1 : 0;
      r[j] = v;
      int t = nt++;
      while (t > 0 && taken[t - 1] > v) {
        taken[t] = taken[t - 1];
        --t;
      }
      taken[t] = v;
    }
    const int64_t base = s * a.P + (k == 3 ? r[0] : a.gbest[s]);
    const int64_t d1 = s * a.P + (k == 3 ? r[1] : r[0]);
    const int64_t d2 = s * a.P + (k == 3 ? r[2] : r[1]);
    const int jr = (int)rng_below(rng_key(pj, (uint64_t)p, 0), (uint32_t)N);
    for (int d = 0; d < N; ++d) {
      double v = __dadd_rn(a.pbx[base * a.nmax + d],
                           __dmul_rn(F, __dsub_rn(a.pbx[d1 * a.nmax + d], a.pbx[d2 * a.nmax + d])));
      if (v < lo || v > hi) v = __dadd_rn(lo, __dmul_rn(span, rng_uniform(pb, (uint64_t)p, (uint64_t)d)));
      const bool take = rng_uniform(pcr, (uint64_t)p, (uint64_t)d) < a.de_cr || d == jr;
      a.x[q * a.nmax + d] = take ? v : a.pbx[q * a.nmax + d];
    }
  }
}

// ------------------------------------------------------------------ dual annealing
// Generalized simulated annealing chains (Tsallis and Stariolo), one per member:
// current state in cx/ce, best state in pbx/pbc, trial states written to x for
// evaluation. Outer iteration t (the device generation counter) has visiting
// temperature T(t) = T0 (2^(qv-1) - 1) / ((1+t)^(qv-1) - 1) and acceptance
// temperature T(t)/t; its Markov chain has 2N moves, move j < N displacing every
// coordinate and move j >= N coordinate j - N, by dx = sigma(T) z1 / |z2|^a with
// a = (qv-1)/(3-qv), sigma(T) = exp((log T - C_QV) / (3-qv)) and (z1, z2) a
// polar-method normal pair (capped at |dx| <= 1e8), wrapped periodically into
// [lo, hi]. A lower energy is accepted; a higher one with probability
// [1 - (1-qa) dE / T_acc]^(1/(1-qa)) against a uniform draw. All arithmetic is
// explicit __d*_rn and the fixed-operation log/exp, so the chains are
// bit-identical to an FP64 implementation of the same sequence.
constexpr double DA_QV = 2.62;
constexpr double DA_C_QV = -0.6233798028078907;  // (qv-1) log(A/B) at qv = 2.62 (40-digit evaluation)
constexpr double DA_TAIL = 1.0e8;
constexpr int DA_NMAX_SLOTS = 20;                // slot stride per move (pole capacity)

__device__ __forceinline__ double da_temperature(double t0, int t) {
  const double num = __dsub_rn(dm_exp(__dmul_rn(__dsub_rn(DA_QV, 1.0), dm_log(2.0))), 1.0);
  const double den = __dsub_rn(dm_exp(__dmul_rn(__dsub_rn(DA_QV, 1.0), dm_log(__dadd_rn((double)t, 1.0)))), 1.0);
  return __ddiv_rn(__dmul_rn(t0, num), den);
}

// Copy the evaluated initial members into the chains' current states.
__global__ void k_da_start(SwarmArgs a) {
  const int64_t Q = (int64_t)a.S * a.P;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
       q += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < a.nmax; ++d) a.cx[q * a.nmax + d] = a.pbx[q * a.nmax + d];
    a.ce[q] = a.pbc[q];
  }
}

__global__ void k_da_visit(SwarmArgs a, int j) {
  const int64_t Q = (int64_t)a.S * a.P;
  const int t = *a.gen;
  const double T = da_temperature(a.da_t0, t);
  const double sig = dm_exp(__ddiv_rn(__dsub_rn(dm_log(T), DA_C_QV), __dsub_rn(3.0, DA_QV)));
  const double pw = __ddiv_rn(__dsub_rn(DA_QV, 1.0), __dsub_rn(3.0, DA_QV));
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / a.P;
    const int p = (int)(q % a.P);
    const int N = a.n_poles[s];
    if (j >= 2 * N) {
      a.active[q] = 0;
      continue;
    }
    a.active[q] = 1;
    const double lo = a.lo[s], hi = a.hi[s], span = __dsub_rn(hi, lo);
    const uint64_t pv = rng_prefix(a.seed, TAG_DA_VISIT, key_id(a, s), (uint64_t)t);
    const int d0 = j < N ? 0 : j - N, d1 = j < N ? N : j - N + 1;
    for (int d = 0; d < a.nmax; ++d) {
      double xv = a.cx[q * a.nmax + d];
      if (d >= d0 && d < d1) {
        double z1 = 0.0, z2 = 0.0;
        for (int k = 0; k < DM_POLAR_TRIES; ++k) {
          const uint64_t slot = ((uint64_t)(j * DA_NMAX_SLOTS + d) * DM_POLAR_TRIES + k) * 2;
          const double u = __dsub_rn(__dmul_rn(2.0, rng_uniform(pv, (uint64_t)p, slot)), 1.0);
          const double v = __dsub_rn(__dmul_rn(2.0, rng_uniform(pv, (uint64_t)p, slot + 1)), 1.0);
          const double ss = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
          if (ss > 0.0 && ss < 1.0) {
            const double f = __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, dm_log(ss)), ss));
            z1 = __dmul_rn(u, f);
            z2 = __dmul_rn(v, f);
            break;
          }
        }
        const double az = fabs(z2);
        double dx;
        if (az > 0.0) dx = __ddiv_rn(__dmul_rn(sig, z1), dm_exp(__dmul_rn(pw, dm_log(az))));
        else dx = copysign(DA_TAIL, z1);
        dx = fmin(fmax(dx, -DA_TAIL), DA_TAIL);
        xv = __dadd_rn(xv, dx);
        if (xv < lo || xv > hi) {
          double r = fmod(__dsub_rn(xv, lo), span);
          if (r < 0.0) r = __dadd_rn(r, span);
          xv = __dadd_rn(lo, r);
        }
      }
      a.x[q * a.nmax + d] = xv;
    }
  }
}

__global__ void k_da_accept(SwarmArgs a, const double* __restrict__ cost, int j) {
  const int64_t Q = (int64_t)a.S * a.P;
  const int t = *a.gen;
  const double T = da_temperature(a.da_t0, t);
  const double t_acc = __ddiv_rn(T, (double)t);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / a.P;
    const int p = (int)(q % a.P);
    const int N = a.n_poles[s];
    if (j >= 2 * N) continue;
    double et = cost[q];
    if (!isfinite(et)) et = INFINITY;
    const double e = a.ce[q];
    bool acc = et < e;
    if (!acc && isfinite(et)) {
      const double tmp = __dsub_rn(1.0, __ddiv_rn(__dmul_rn(__dsub_rn(1.0, a.da_qa), __dsub_rn(et, e)), t_acc));
      const double pr = tmp > 0.0 ? dm_exp(__ddiv_rn(dm_log(tmp), __dsub_rn(1.0, a.da_qa))) : 0.0;
      const double u = rng_uniform(rng_prefix(a.seed, TAG_DA_ACCEPT, key_id(a, s), (uint64_t)t), (uint64_t)p,
                                   (uint64_t)j);
      acc = u <= pr;
    }
    if (!acc) continue;
    for (int d = 0; d < N; ++d) a.cx[q * a.nmax + d] = a.x[q * a.nmax + d];
    a.ce[q] = et;
    if (et < a.pbc[q]) {
      for (int d = 0; d < N; ++d) a.pbx[q * a.nmax + d] = a.x[q * a.nmax + d];
      a.pbc[q] = et;
    }
  }
}

// Lexicographic (cost, index) minimum: lowest cost, lowest index on ties.
__device__ __forceinline__ void argmin_merge(double& c, int& i, double c2, int i2) {
  if (c2 < c || (c2 == c && i2 < i)) {
    c = c2;
    i = i2;
  }
}

__device__ __forceinline__ void block_argmin(double& c, int& i) {
  __shared__ double sc[32];
  __shared__ int si[32];
  for (int o = 16; o > 0; o >>= 1) {
    const double c2 = __shfl_down_sync(0xffffffffu, c, o);
    const int i2 = __shfl_down_sync(0xffffffffu, i, o);
    argmin_merge(c, i, c2, i2);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sc[wid] = c;
    si[wid] = i;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    c = lane < nw ? sc[lane] : INFINITY;
    i = lane < nw ? si[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double c2 = __shfl_down_sync(0xffffffffu, c, o);
      const int i2 = __shfl_down_sync(0xffffffffu, i, o);
      argmin_merge(c, i, c2, i2);
    }
  }
  __syncthreads();
}

// Personal bests (strictly lower cost replaces; generation 0 initialises) and
// the global best per spectrum; one block per spectrum.
__global__ void k_pso_best(SwarmArgs a, const double* __restrict__ cost) {
  const int gen = *a.gen;
  for (int64_t s = blockIdx.x; s < a.S; s += gridDim.x) {
    const int N = a.n_poles[s];
    double bc = INFINITY;
    int bi = 0x7fffffff;
    for (int p = threadIdx.x; p < a.P; p += blockDim.x) {
      const int64_t q = s * a.P + p;
      double c = cost[q];
      if (!isfinite(c)) c = INFINITY;
      double pc = a.pbc[q];
      if (gen == 0 || c < pc) {
        pc = c;
        a.pbc[q] = c;
        for (int d = 0; d < N; ++d) a.pbx[q * a.nmax + d] = a.x[q * a.nmax + d];
      }
      argmin_merge(bc, bi, pc, p);
    }
    block_argmin(bc, bi);
    if (threadIdx.x == 0) {
      a.gbest[s] = bi < a.P ? bi : 0;
      if (a.trace) a.trace[s * (int64_t)(a.iters + 1) + gen] = bc;
      if (a.evals) atomicAdd(a.evals, (double)a.P * (double)(a.offsets[s + 1] - a.offsets[s]));
    }
  }
}

// After an outer iteration of dual annealing: best chain per spectrum (lowest
// best cost, lowest index on ties), its cost in the trace, and the iteration's
// evaluations (P chains x 2N moves x K samples) in the counter.
__global__ void k_da_best(SwarmArgs a) {
  const int gen = *a.gen;
  for (int64_t s = blockIdx.x; s < a.S; s += gridDim.x) {
    double bc = INFINITY;
    int bi = 0x7fffffff;
    for (int p = threadIdx.x; p < a.P; p += blockDim.x) argmin_merge(bc, bi, a.pbc[s * a.P + p], p);
    block_argmin(bc, bi);
    if (threadIdx.x == 0) {
      a.gbest[s] = bi < a.P ? bi : 0;
      if (a.trace) a.trace[s * (int64_t)(a.iters + 1) + gen] = bc;
      if (a.evals)
        atomicAdd(a.evals, (double)a.P * 2.0 * (double)a.n_poles[s] * (double)(a.offsets[s + 1] - a.offsets[s]));
    }
  }
}

__global__ void k_gen_advance(int* gen) { *gen += 1; }

__global__ void k_add_scalar(double* dst, double v) { *dst += v; }

// ------------------------------------------------------------------ top-k and polish
// Lines l = s * T + j start from the j-th best personal best of spectrum s.
__global__ void k_topk(SwarmArgs a, PolishArgs pa) {
  extern __shared__ unsigned char taken_raw[];
  unsigned char* taken = taken_raw;
  for (int64_t s = blockIdx.x; s < a.S; s += gridDim.x) {
    for (int p = threadIdx.x; p < a.P; p += blockDim.x) taken[p] = 0;
    __syncthreads();
    for (int j = 0; j < pa.T; ++j) {
      double bc = INFINITY;
      int bi = 0x7fffffff;
      for (int p = threadIdx.x; p < a.P; p += blockDim.x)
        if (!taken[p]) argmin_merge(bc, bi, a.pbc[s * a.P + p], p);
      block_argmin(bc, bi);
      if (threadIdx.x == 0) {
        const int p = bi < a.P ? bi : 0;
        taken[p] = 1;
        const int64_t l = s * pa.T + j;
        for (int d = 0; d < a.nmax; ++d) pa.th[l * a.nmax + d] = a.pbx[(s * a.P + p) * a.nmax + d];
        pa.f[l] = bc;
        pa.done[l] = 0;
        pa.hcount[l] = 0;
      }
      __syncthreads();
    }
  }
}

// The start point of each line is evaluated, with its gradient, in the
// accepted-point slot (candidate l of the gradient evaluation).
__global__ void k_polish_start(PolishArgs pa) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pa.L;
       l += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < pa.nmax; ++d) pa.ath[l * pa.nmax + d] = pa.th[l * pa.nmax + d];
    pa.aactive[l] = 1;
    for (int t = 0; t < pa.R; ++t) pa.active[l * pa.R + t] = 0;
  }
}

// After the start evaluation: f, g of each line.
__global__ void k_polish_take0(PolishArgs pa) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pa.L;
       l += (int64_t)gridDim.x * blockDim.x) {
    pa.f[l] = pa.acost[l];
    for (int d = 0; d < pa.nmax; ++d) pa.g[l * pa.nmax + d] = pa.agrad[l * pa.nmax + d];
    pa.aactive[l] = 0;
    if (!isfinite(pa.f[l])) pa.done[l] = 1;
  }
}

__device__ __forceinline__ double dotn(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = fma(a[i], b[i], s);
  return s;
}

__device__ void write_trials(const PolishArgs& pa, int64_t l, int N, double lo, double hi) {
  const int nmax = pa.nmax;
  const int t0 = pa.t0[l];
  for (int t = 0; t < pa.R; ++t) {
    const int64_t q = l * pa.R + t;
    const int tt = t0 + t;
    if (tt >= pa.max_trials) {
      pa.active[q] = 0;
      continue;
    }
    const double step = ldexp(1.0, -tt);
    for (int d = 0; d < nmax; ++d) {
      double v = 0.0;
      if (d < N) v = fmin(fmax(pa.th[l * nmax + d] + step * pa.dir[l * nmax + d], lo), hi);
      pa.tth[q * nmax + d] = v;
    }
    pa.active[q] = 1;
  }
}

// Two-loop recursion (Nocedal and Wright, Alg. 7.4) for the direction d = -H g;
// a non-descent direction is replaced by -g / max(1, |g|_inf) and the history cleared.
__global__ void k_polish_dir(PolishArgs pa, const int32_t* n_poles, const double* lo_, const double* hi_) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pa.L;
       l += (int64_t)gridDim.x * blockDim.x) {
    pa.acc[l] = 0;
    if (pa.done[l]) continue;
    const int64_t s = l / pa.T;
    const int N = n_poles[s];
    const int nmax = pa.nmax, m = pa.m;
    double q[NMAX], alpha[8];
    const double* g = pa.g + l * nmax;
    for (int d = 0; d < N; ++d) q[d] = g[d];
    const int hc = pa.hcount[l];
    // history slot of the k-th newest pair: (head - 1 - k) mod m, head = hc mod m ... stored oldest..newest
    for (int k = hc - 1; k >= 0; --k) {
      const double* sk = pa.hs + (l * m + k) * nmax;
      const double* yk = pa.hy + (l * m + k) * nmax;
      const double rho = 1.0 / dotn(yk, sk, N);
      const double al = rho * dotn(sk, q, N);
      for (int d = 0; d < N; ++d) q[d] -= al * yk[d];
      alpha[k] = al;
    }
    double gamma;
    if (hc > 0) {
      const double* sn = pa.hs + (l * m + hc - 1) * nmax;
      const double* yn = pa.hy + (l * m + hc - 1) * nmax;
      gamma = dotn(sn, yn, N) / dotn(yn, yn, N);
    } else {
      double gi = 0.0;
      for (int d = 0; d < N; ++d) gi = fmax(gi, fabs(g[d]));
      gamma = 1.0 / fmax(1.0, gi);
    }
    for (int d = 0; d < N; ++d) q[d] *= gamma;
    for (int k = 0; k < hc; ++k) {
      const double* sk = pa.hs + (l * m + k) * nmax;
      const double* yk = pa.hy + (l * m + k) * nmax;
      const double rho = 1.0 / dotn(yk, sk, N);
      const double be = rho * dotn(yk, q, N);
      for (int d = 0; d < N; ++d) q[d] += sk[d] * (alpha[k] - be);
    }
    double gd = 0.0;
    for (int d = 0; d < N; ++d) gd = fma(g[d], -q[d], gd);
    double* dir = pa.dir + l * nmax;
    if (!(gd < 0.0)) {
      double gi = 0.0;
      for (int d = 0; d < N; ++d) gi = fmax(gi, fabs(g[d]));
      const double sc = 1.0 / fmax(1.0, gi);
      for (int d = 0; d < N; ++d) dir[d] = -g[d] * sc;
      pa.hcount[l] = 0;
    } else {
      for (int d = 0; d < N; ++d) dir[d] = -q[d];
    }
    // the full step t = 0 is evaluated first, with its gradient, in the accepted-point slot;
    // the backtracking rounds start at t = 1 if it fails
    for (int d = 0; d < nmax; ++d) {
      double v = 0.0;
      if (d < N) v = fmin(fmax(pa.th[l * nmax + d] + dir[d], lo_[s]), hi_[s]);
      pa.ath[l * nmax + d] = v;
    }
    pa.aactive[l] = 1;
    pa.t0[l] = 1;
  }
}

// Armijo test of the full step (evaluated with its gradient in the accepted-point
// slot): accepted, the line's cost and gradient are ready for the update; rejected,
// the backtracking trials t = 1 .. R of the first round are written.
__global__ void k_polish_first(PolishArgs pa, const int32_t* n_poles, const double* lo_, const double* hi_,
                               const int64_t* offsets) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pa.L;
       l += (int64_t)gridDim.x * blockDim.x) {
    if (!pa.aactive[l]) continue;
    pa.aactive[l] = 0;
    const int64_t s = l / pa.T;
    const int N = n_poles[s];
    const int nmax = pa.nmax;
    if (pa.evals) atomicAdd(pa.evals, (double)(offsets[s + 1] - offsets[s]));
    double gs = 0.0;
    for (int d = 0; d < N; ++d) gs = fma(pa.g[l * nmax + d], pa.ath[l * nmax + d] - pa.th[l * nmax + d], gs);
    if (pa.acost[l] <= pa.f[l] + pa.c1 * gs) {
      pa.acc[l] = 1;
    } else if (pa.t0[l] >= pa.max_trials) {
      pa.done[l] = 1;
    } else {
      write_trials(pa, l, N, lo_[s], hi_[s]);
    }
  }
}

// Armijo test on the evaluated trials of each line, in order of decreasing step.
__global__ void k_polish_accept(PolishArgs pa, const int32_t* n_poles, const double* lo_, const double* hi_,
                                const int64_t* offsets) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pa.L;
       l += (int64_t)gridDim.x * blockDim.x) {
    if (pa.done[l] || pa.acc[l]) continue;
    const int64_t s = l / pa.T;
    const int N = n_poles[s];
    const int nmax = pa.nmax;
    int n_active = 0;
    int hit = -1;
    for (int t = 0; t < pa.R; ++t) {
      const int64_t q = l * pa.R + t;
      if (!pa.active[q]) continue;
      ++n_active;
      if (hit >= 0) continue;
      double gs = 0.0;
      for (int d = 0; d < N; ++d)
        gs = fma(pa.g[l * nmax + d], pa.tth[q * nmax + d] - pa.th[l * nmax + d], gs);
      if (pa.tcost[q] <= pa.f[l] + pa.c1 * gs) hit = t;
    }
    // the trials a sequential backtracking search evaluates: up to and including the first
    // acceptable one (the speculative trials after it are not counted)
    const int counted = hit >= 0 ? hit + 1 : n_active;
    if (pa.evals && counted) atomicAdd(pa.evals, (double)counted * (double)(offsets[s + 1] - offsets[s]));
    for (int t = 0; t < pa.R; ++t) pa.active[l * pa.R + t] = 0;
    if (hit >= 0) {
      const int64_t q = l * pa.R + hit;
      for (int d = 0; d < nmax; ++d) pa.ath[l * nmax + d] = pa.tth[q * nmax + d];
      pa.aactive[l] = 1;
      pa.acc[l] = 1;
    } else if (n_active) {
      pa.t0[l] += pa.R;
      if (pa.t0[l] >= pa.max_trials) pa.done[l] = 1;
      else write_trials(pa, l, N, lo_[s], hi_[s]);
    }
  }
}

// L-BFGS update with the accepted point's cost and gradient: history pair
// (s, y) kept only when s^T y > eps y^T y (oldest pair dropped when full).
__global__ void k_polish_take(PolishArgs pa, const int32_t* n_poles) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < pa.L;
       l += (int64_t)gridDim.x * blockDim.x) {
    if (!pa.acc[l]) continue;
    pa.aactive[l] = 0;
    const int64_t s = l / pa.T;
    const int N = n_poles[s];
    const int nmax = pa.nmax, m = pa.m;
    double sv[NMAX], yv[NMAX];
    for (int d = 0; d < N; ++d) {
      sv[d] = pa.ath[l * nmax + d] - pa.th[l * nmax + d];
      yv[d] = pa.agrad[l * nmax + d] - pa.g[l * nmax + d];
    }
    const double sy = dotn(sv, yv, N), yy = dotn(yv, yv, N);
    if (sy > 2.220446049250313e-16 * yy) {
      int hc = pa.hcount[l];
      if (hc == m) {
        for (int k = 1; k < m; ++k)
          for (int d = 0; d < N; ++d) {
            pa.hs[(l * m + k - 1) * nmax + d] = pa.hs[(l * m + k) * nmax + d];
            pa.hy[(l * m + k - 1) * nmax + d] = pa.hy[(l * m + k) * nmax + d];
          }
        hc = m - 1;
      }
      for (int d = 0; d < N; ++d) {
        pa.hs[(l * m + hc) * nmax + d] = sv[d];
        pa.hy[(l * m + hc) * nmax + d] = yv[d];
      }
      pa.hcount[l] = hc + 1;
    }
    for (int d = 0; d < N; ++d) {
      pa.th[l * nmax + d] = pa.ath[l * nmax + d];
      pa.g[l * nmax + d] = pa.agrad[l * nmax + d];
    }
    pa.f[l] = pa.acost[l];
    if (!isfinite(pa.f[l])) pa.done[l] = 1;
  }
}

// Best line per spectrum (lowest cost, lowest rank on ties), or the swarm's
// global best when there is no polish; writes theta* of spectrum s to out[s].
__global__ void k_pick_best(SwarmArgs a, PolishArgs pa, double* out_theta) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < a.S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const double* src;
    if (pa.T > 0) {
      double bc = INFINITY;
      int bj = 0x7fffffff;
      for (int j = 0; j < pa.T; ++j) argmin_merge(bc, bj, pa.f[s * pa.T + j], j);
      if (bj >= pa.T) bj = 0;
      src = pa.th + (s * pa.T + bj) * a.nmax;
    } else {
      src = a.pbx + (s * a.P + a.gbest[s]) * a.nmax;
    }
    for (int d = 0; d < a.nmax; ++d) out_theta[s * a.nmax + d] = src[d];
  }
}

// Poles sorted by ascending tau (stable), padded with zeros (Listing 2 layout).
__global__ void k_assemble(int64_t S, int nmax, const int32_t* n_poles, const double* theta,
                           const double* weights, const double* cost, double* eps_inf, double* d_eps,
                           double* tau, double* final_cost) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int N = n_poles[s];
    int idx[NMAX];
    for (int i = 0; i < N; ++i) idx[i] = i;
    for (int i = 1; i < N; ++i) {
      const int v = idx[i];
      int j = i - 1;
      while (j >= 0 && theta[s * nmax + idx[j]] > theta[s * nmax + v]) {
        idx[j + 1] = idx[j];
        --j;
      }
      idx[j + 1] = v;
    }
    eps_inf[s] = weights[s * (nmax + 1)];
    for (int i = 0; i < nmax; ++i) {
      if (i < N) {
        d_eps[s * nmax + i] = weights[s * (nmax + 1) + 1 + idx[i]];
        tau[s * nmax + i] = exp10(theta[s * nmax + idx[i]]);
      } else {
        d_eps[s * nmax + i] = 0.0;
        tau[s * nmax + i] = 0.0;
      }
    }
    final_cost[s] = cost[s];
  }
}

// ------------------------------------------------------------------ launchers
static int g1d(int64_t n, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8)); }
// Grid for one thread per item in blocks of `block` threads (at most 2048 resident per SM).
static int g1d_b(int64_t n, int block, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + block - 1) / block, (int64_t)sms * (2048 / block)));
}
// The polish's per-line kernels run one thread per line through a dependent FP64
// chain (the L-BFGS two-loop recursion, the Armijo tests): single-warp blocks spread
// the lines over every SM.
constexpr int POLISH_BLOCK = 32;

void launch_pso_init(const SwarmArgs& a, int sms, cudaStream_t st) {
  k_pso_init<<<g1d((int64_t)a.S * a.P, sms), 256, 0, st>>>(a);
}
void launch_pso_move(const SwarmArgs& a, int sms, cudaStream_t st) {
  k_pso_move<<<g1d((int64_t)a.S * a.P, sms), 256, 0, st>>>(a);
}
void launch_de_trial(const SwarmArgs& a, int sms, cudaStream_t st) {
  k_de_trial<<<g1d((int64_t)a.S * a.P, sms), 256, 0, st>>>(a);
}
void launch_da_start(const SwarmArgs& a, int sms, cudaStream_t st) {
  k_da_start<<<g1d((int64_t)a.S * a.P, sms), 256, 0, st>>>(a);
}
void launch_da_visit(const SwarmArgs& a, int j, int sms, cudaStream_t st) {
  k_da_visit<<<g1d_b((int64_t)a.S * a.P, 128, sms), 128, 0, st>>>(a, j);
}
void launch_da_accept(const SwarmArgs& a, const double* cost, int j, int sms, cudaStream_t st) {
  k_da_accept<<<g1d((int64_t)a.S * a.P, sms), 256, 0, st>>>(a, cost, j);
}
void launch_da_best(const SwarmArgs& a, int sms, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.S, (int64_t)sms * 8));
  k_da_best<<<grid, 256, 0, st>>>(a);
}
void launch_pso_best(const SwarmArgs& a, const double* cost, int sms, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.S, (int64_t)sms * 8));
  k_pso_best<<<grid, 256, 0, st>>>(a, cost);
}
void launch_gen_advance(int* gen, cudaStream_t st) { k_gen_advance<<<1, 1, 0, st>>>(gen); }
void launch_add_scalar(double* dst, double v, cudaStream_t st) { k_add_scalar<<<1, 1, 0, st>>>(dst, v); }
void launch_topk(const SwarmArgs& a, const PolishArgs& pa, int sms, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.S, (int64_t)sms * 8));
  k_topk<<<grid, 256, a.P, st>>>(a, pa);
}
void launch_polish_start(const PolishArgs& pa, int sms, cudaStream_t st) {
  k_polish_start<<<g1d(pa.L, sms), 256, 0, st>>>(pa);
}
void launch_polish_take0(const PolishArgs& pa, int sms, cudaStream_t st) {
  k_polish_take0<<<g1d(pa.L, sms), 256, 0, st>>>(pa);
}
void launch_polish_dir(const PolishArgs& pa, const int32_t* n_poles, const double* lo, const double* hi,
                       int sms, cudaStream_t st) {
  k_polish_dir<<<g1d_b(pa.L, POLISH_BLOCK, sms), POLISH_BLOCK, 0, st>>>(pa, n_poles, lo, hi);
}
void launch_polish_first(const PolishArgs& pa, const int32_t* n_poles, const double* lo, const double* hi,
                         const int64_t* offsets, int sms, cudaStream_t st) {
  k_polish_first<<<g1d_b(pa.L, POLISH_BLOCK, sms), POLISH_BLOCK, 0, st>>>(pa, n_poles, lo, hi, offsets);
}
void launch_polish_accept(const PolishArgs& pa, const int32_t* n_poles, const double* lo, const double* hi,
                          const int64_t* offsets, int sms, cudaStream_t st) {
  k_polish_accept<<<g1d_b(pa.L, POLISH_BLOCK, sms), POLISH_BLOCK, 0, st>>>(pa, n_poles, lo, hi, offsets);
}
void launch_polish_take(const PolishArgs& pa, const int32_t* n_poles, int sms, cudaStream_t st) {
  k_polish_take<<<g1d_b(pa.L, POLISH_BLOCK, sms), POLISH_BLOCK, 0, st>>>(pa, n_poles);
}
void launch_pick_best(const SwarmArgs& a, const PolishArgs& pa, double* out_theta, int sms, cudaStream_t st) {
  k_pick_best<<<g1d(a.S, sms), 256, 0, st>>>(a, pa, out_theta);
}
void launch_assemble(int64_t S, int nmax, const int32_t* n_poles, const double* theta, const double* weights,
                     const double* cost, double* eps_inf, double* d_eps, double* tau, double* final_cost,
                     int sms, cudaStream_t st) {
  k_assemble<<<g1d(S, sms), 256, 0, st>>>(S, nmax, n_poles, theta, weights, cost, eps_inf, d_eps, tau,
                                           final_cost);
}

}  // namespace debyefit
