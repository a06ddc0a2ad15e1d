// debye_fit_auto: automatic number of poles (Sec. III-B, "N = -1").
//
// The paper grows N from one pole until the fit's error is below 5 % or N
// reaches 20. Each N is a complete, independent fit, so the fits for several N
// can run together: work proceeds in waves of `wave` consecutive pole counts,
// every spectrum still looking for its N contributes one virtual spectrum per
// pole count of the wave (a copy of its samples with that N), and the whole
// wave is one ragged debye_fit_batch run. The generator's keys use the original
// spectrum index, so every fit equals the one a sequential N = 1, 2, ... loop
// would make. After a wave, each spectrum takes the first N of the wave whose
// average fractional error (Sec. IV: mean relative error of eps' plus that of
// eps'', in percent) is below the threshold, or its cap; spectra that found
// their N leave the next wave.
#include <algorithm>
#include <cmath>
#include <vector>

#include "host.h"
#include "search.h"

namespace debyefit {
namespace {

// Virtual spectrum v gets the samples and bounds of spectrum src[v].
__global__ void k_expand(int64_t V, const int64_t* __restrict__ src, const int64_t* __restrict__ voffs,
                         const int64_t* __restrict__ offs, const double* __restrict__ omega,
                         const double* __restrict__ er, const double* __restrict__ ei,
                         const double* __restrict__ lo, const double* __restrict__ hi, double* vomega,
                         double* ver, double* vei, double* vlo, double* vhi, int* status) {
  for (int64_t v = blockIdx.x; v < V; v += gridDim.x) {
    const int64_t s = src[v], a = offs[s], b = voffs[v];
    const int64_t n = voffs[v + 1] - b;
    if (offs[s + 1] - a != n) {  // host and device offsets disagree
      if (threadIdx.x == 0) atomicCAS(status, 0, DEBYE_EBOUNDS);
      continue;
    }
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
      vomega[b + k] = omega[a + k];
      ver[b + k] = er[a + k];
      vei[b + k] = ei[a + k];
    }
    if (threadIdx.x == 0) {
      vlo[v] = lo[s];
      vhi[v] = hi[s];
    }
  }
}

// Average fractional error (percent) of every virtual spectrum's fit: one block each.
__global__ void k_frac_err(int64_t V, const int64_t* __restrict__ voffs, const double* __restrict__ omega,
                           const double* __restrict__ er, const double* __restrict__ ei,
                           const int32_t* __restrict__ vn, int nmaxw, const double* __restrict__ eps_inf,
                           const double* __restrict__ d_eps, const double* __restrict__ tau, double* err) {
  __shared__ double sr[32], si[32];
  for (int64_t v = blockIdx.x; v < V; v += gridDim.x) {
    const int N = vn[v];
    const int64_t a = voffs[v], K = voffs[v + 1] - a;
    double accr = 0.0, acci = 0.0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
      const double w = omega[a + k];
      double fr = eps_inf[v], fi = 0.0;
      for (int n = 0; n < N; ++n) {
        const double x = w * tau[v * nmaxw + n];
        const double den = 1.0 + x * x;
        fr += d_eps[v * nmaxw + n] / den;
        fi += d_eps[v * nmaxw + n] * x / den;
      }
      accr += fabs(fr - er[a + k]) / fabs(er[a + k]);
      acci += fabs(fi - ei[a + k]) / fabs(ei[a + k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      accr += __shfl_down_sync(0xffffffffu, accr, o);
      acci += __shfl_down_sync(0xffffffffu, acci, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      sr[wid] = accr;
      si[wid] = acci;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0, i = 0.0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
        r += sr[j];
        i += si[j];
      }
      err[v] = 100.0 * (r / (double)K + i / (double)K);
    }
    __syncthreads();
  }
}

// For every spectrum of the wave: the first virtual fit (ascending N) whose error is
// below the threshold, or the one at the spectrum's cap; its result becomes the output.
__global__ void k_auto_pick(int64_t A, const int64_t* __restrict__ act_s, const int64_t* __restrict__ act_vb,
                            const int64_t* __restrict__ act_ve, const int32_t* __restrict__ vn,
                            const int32_t* __restrict__ ncap, double thr, const double* __restrict__ verr,
                            const double* __restrict__ v_eps_inf, const double* __restrict__ v_deps,
                            const double* __restrict__ v_tau, const double* __restrict__ v_cost, int nmaxw,
                            int nmax, double* eps_inf, double* d_eps, double* tau, double* final_cost,
                            double* frac_err, int32_t* n_chosen, int32_t* done) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = act_s[i];
    int64_t c = -1;
    for (int64_t v = act_vb[i]; v < act_ve[i]; ++v) {
      if (verr[v] < thr || vn[v] >= ncap[s]) {
        c = v;
        break;
      }
    }
    if (c < 0) continue;
    const int N = vn[c];
    eps_inf[s] = v_eps_inf[c];
    for (int n = 0; n < nmax; ++n) {
      d_eps[s * nmax + n] = n < N ? v_deps[c * nmaxw + n] : 0.0;
      tau[s * nmax + n] = n < N ? v_tau[c * nmaxw + n] : 0.0;
    }
    final_cost[s] = v_cost[c];
    frac_err[s] = verr[c];
    n_chosen[s] = N;
    done[s] = 1;
  }
}

int grid_for(int64_t n, int per_block, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, (int64_t)sms * 8));
}

}  // namespace
}  // namespace debyefit

using namespace debyefit;

extern "C" int debye_fit_auto(debye_handle h, const debye_spectra* sp, const debye_search* se, int32_t n_max,
                              double threshold, int32_t wave, double* eps_inf, double* d_eps, double* tau,
                              double* final_cost, double* frac_err, int32_t* n_chosen, cudaStream_t st) {
  if (!h) return DEBYE_EINVAL;
  h->err.clear();
  if (!sp || !se) return h->fail(DEBYE_EINVAL, "spectra or search is NULL");
  if (se->trace) return h->fail(DEBYE_EINVAL, "search->trace is not supported by debye_fit_auto");
  if (se->n_failed) return h->fail(DEBYE_EINVAL, "search->n_failed is not supported by debye_fit_auto");
  if (se->P < 1 || se->P > 32768) return h->fail(DEBYE_EINVAL, "P = %d outside 1..32768", se->P);
  if (se->iters < 0 || se->polish_iters < 0) return h->fail(DEBYE_EINVAL, "iters < 0 or polish_iters < 0");
  if (se->polish_topk < 0 || se->polish_topk > 64) return h->fail(DEBYE_EINVAL, "polish_topk outside 0..64");
  if (se->method != DEBYE_SEARCH_PSO && se->method != DEBYE_SEARCH_DE && se->method != DEBYE_SEARCH_DA)
    return h->fail(DEBYE_EINVAL, "method must be DEBYE_SEARCH_PSO, DEBYE_SEARCH_DE or DEBYE_SEARCH_DA");
  if (se->method == DEBYE_SEARCH_DA && se->iters > 1000)
    return h->fail(DEBYE_EINVAL, "dual annealing: at most 1000 outer iterations");
  if (se->method == DEBYE_SEARCH_DE && se->iters > 0 &&
      se->P < (h->opt.de_strategy == DEBYE_DE_RAND1 ? 4 : 3))
    return h->fail(DEBYE_EINVAL, "differential evolution needs P >= %d",
                   h->opt.de_strategy == DEBYE_DE_RAND1 ? 4 : 3);
  if (n_max < 1 || n_max > NMAX) return h->fail(DEBYE_EINVAL, "n_max = %d outside 1..%d", n_max, NMAX);
  if (!(threshold >= 0.0)) return h->fail(DEBYE_EINVAL, "threshold must be >= 0");
  if (wave < 1 || wave > NMAX) return h->fail(DEBYE_EINVAL, "wave = %d outside 1..%d", wave, NMAX);
  if (sp->S > 0 && (!eps_inf || !d_eps || !tau || !final_cost || !frac_err || !n_chosen))
    return h->fail(DEBYE_EINVAL, "an output is NULL");

  cudaStream_t ws = h->work_stream;
  cudaEventRecord(h->ev_in, st);
  cudaStreamWaitEvent(ws, h->ev_in, 0);
  int rc = DEBYE_OK;
  Plan pl;
  auto run = [&]() -> int {
    int r;
    if ((r = h->load_plan(sp, pl, ws))) return r;
    if (pl.nmax_seen > n_max) return h->fail(DEBYE_EINVAL, "n_max = %d < largest cap = %d", n_max, pl.nmax_seen);
    const int64_t S = pl.S;
    if (S == 0) return DEBYE_OK;
    void* p;
    if ((r = h->named("auto.done", sizeof(int32_t) * S, &p))) return r;
    int32_t* d_done = (int32_t*)p;
    cudaMemsetAsync(d_done, 0, sizeof(int32_t) * S, ws);
    std::vector<int32_t> done(S, 0);
    bool first = true;
    for (int n0 = 1; n0 <= pl.nmax_seen; n0 += wave) {
      // the wave's virtual spectra, grouped by spectrum, N ascending
      std::vector<int64_t> vsrc, voffs(1, 0), act_s, act_vb, act_ve;
      std::vector<int32_t> vn;
      int nmaxw = 0;
      for (int64_t s = 0; s < S; ++s) {
        if (done[s] || pl.npol[s] < n0) continue;
        act_s.push_back(s);
        act_vb.push_back((int64_t)vsrc.size());
        for (int N = n0; N < n0 + wave && N <= pl.npol[s]; ++N) {
          vsrc.push_back(s);
          vn.push_back(N);
          voffs.push_back(voffs.back() + (pl.offs[s + 1] - pl.offs[s]));
          nmaxw = std::max(nmaxw, N);
        }
        act_ve.push_back((int64_t)vsrc.size());
      }
      if (act_s.empty()) break;
      const int64_t V = (int64_t)vsrc.size(), A = (int64_t)act_s.size(), KV = voffs.back();
      if (V * (int64_t)se->P > ((int64_t)1 << 31) - 1) return h->fail(DEBYE_EINVAL, "wave too large: reduce wave");
      struct Arr {
        const char* name;
        size_t bytes;
        void** out;
      };
      int64_t *d_vsrc, *d_voffs, *d_act;
      int32_t* d_vn;
      double *vom, *ver, *vei, *vlo, *vhi, *v_inf, *v_deps, *v_tau, *v_cost, *v_err;
      const Arr arrs[] = {
          {"auto.vsrc", sizeof(int64_t) * V, (void**)&d_vsrc},
          {"auto.voffs", sizeof(int64_t) * (V + 1), (void**)&d_voffs},
          {"auto.act", sizeof(int64_t) * 3 * A, (void**)&d_act},
          {"auto.vn", sizeof(int32_t) * V, (void**)&d_vn},
          {"auto.omega", sizeof(double) * KV, (void**)&vom},
          {"auto.re", sizeof(double) * KV, (void**)&ver},
          {"auto.im", sizeof(double) * KV, (void**)&vei},
          {"auto.lo", sizeof(double) * V, (void**)&vlo},
          {"auto.hi", sizeof(double) * V, (void**)&vhi},
          {"auto.v_inf", sizeof(double) * V, (void**)&v_inf},
          {"auto.v_deps", sizeof(double) * V * nmaxw, (void**)&v_deps},
          {"auto.v_tau", sizeof(double) * V * nmaxw, (void**)&v_tau},
          {"auto.v_cost", sizeof(double) * V, (void**)&v_cost},
          {"auto.v_err", sizeof(double) * V, (void**)&v_err},
      };
      for (const Arr& a : arrs)
        if ((r = h->named(a.name, a.bytes, a.out))) return r;
      std::vector<int64_t> act(3 * A);
      std::copy(act_s.begin(), act_s.end(), act.begin());
      std::copy(act_vb.begin(), act_vb.end(), act.begin() + A);
      std::copy(act_ve.begin(), act_ve.end(), act.begin() + 2 * A);
      cudaError_t e = cudaMemcpyAsync(d_vsrc, vsrc.data(), sizeof(int64_t) * V, cudaMemcpyHostToDevice, ws);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_voffs, voffs.data(), sizeof(int64_t) * (V + 1), cudaMemcpyHostToDevice, ws);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_act, act.data(), sizeof(int64_t) * 3 * A, cudaMemcpyHostToDevice, ws);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_vn, vn.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice, ws);
      if (e != cudaSuccess) return h->fail(DEBYE_ECUDA, "wave upload: %s", cudaGetErrorString(e));
      k_expand<<<grid_for(V, 1, h->sms), 256, 0, ws>>>(V, d_vsrc, d_voffs, sp->offsets, sp->omega, sp->eps_re,
                                                       sp->eps_im, sp->lo, sp->hi, vom, ver, vei, vlo, vhi,
                                                       h->d_status);
      ++h->launches;
      if ((r = h->check_launch("auto expand"))) return r;
      debye_spectra vsp{V, d_voffs, vom, ver, vei, d_vn, vlo, vhi, voffs.data(), vn.data()};
      if ((r = fit_impl(h, &vsp, se, nmaxw, v_inf, v_deps, v_tau, v_cost, ws, d_vsrc, first))) return r;
      first = false;
      k_frac_err<<<grid_for(V, 1, h->sms), 256, 0, ws>>>(V, d_voffs, vom, ver, vei, d_vn, nmaxw, v_inf, v_deps,
                                                         v_tau, v_err);
      ++h->launches;
      k_auto_pick<<<grid_for(A, 128, h->sms), 128, 0, ws>>>(A, d_act, d_act + A, d_act + 2 * A, d_vn, sp->n_poles,
                                                            threshold, v_err, v_inf, v_deps, v_tau, v_cost, nmaxw,
                                                            n_max, eps_inf, d_eps, tau, final_cost, frac_err,
                                                            n_chosen, d_done);
      ++h->launches;
      if ((r = h->check_launch("auto pick"))) return r;
      // which spectra found their N (the host vectors above stay alive until this sync)
      e = cudaMemcpyAsync(done.data(), d_done, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, ws);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ws);
      if (e != cudaSuccess) return h->fail(DEBYE_ECUDA, "wave result: %s", cudaGetErrorString(e));
    }
    return DEBYE_OK;
  };
  rc = run();
  cudaEventRecord(h->ev_out, ws);
  cudaStreamWaitEvent(st, h->ev_out, 0);
  return rc;
}
