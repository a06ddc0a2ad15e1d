// debye_fit_batch: seeded swarm or differential evolution + polish + final
// re-solve (host orchestration).
//
// The work runs on the handle's own non-blocking stream, joined to the
// caller's stream by events, so that the generation loop and the polish loop can
// be captured as CUDA graphs even when the caller uses the legacy default stream.
// One generation (move, evaluate, personal/global bests, counter advance) is
// captured once and launched `iters` times; the generation index lives on the
// device. One polish iteration is captured the same way.
#include <algorithm>
#include <cstring>
#include <vector>

#include "host.h"
#include "search.h"

using namespace debyefit;

namespace {

// Line search of the polish: the full step is evaluated first (with its gradient);
// a line that rejects it evaluates POLISH_R further step lengths per backtracking round.
constexpr int POLISH_R = 8;

struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  ~GraphGuard() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
  }
};

}  // namespace

int debye_ctx::named(const char* name, size_t bytes, void** out) {
  Buf& b = named_bufs[name];
  int rc = ensure(b, bytes, name);
  *out = b.p;
  return rc;
}

// Run `body` `times` times on stream st, captured once as a graph when enabled.
template <class F>
static int repeat(debye_ctx* h, int times, cudaStream_t st, F body) {
  if (times <= 0) return DEBYE_OK;
  if (!h->opt.use_graphs || h->prof_on || times == 1) {
    for (int i = 0; i < times; ++i) {
      int rc = body();
      if (rc) return rc;
    }
    return DEBYE_OK;
  }
  GraphGuard gg;
  const int64_t before = h->launches;
  h->capturing_stream = st;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    h->capturing_stream = nullptr;
    return h->fail(DEBYE_ECUDA, "begin capture: %s", cudaGetErrorString(e));
  }
  int rc = body();
  e = cudaStreamEndCapture(st, &gg.g);
  h->capturing_stream = nullptr;
  if (rc) return rc;
  if (e != cudaSuccess) return h->fail(DEBYE_ECUDA, "end capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&gg.e, gg.g, 0);
  if (e != cudaSuccess) return h->fail(DEBYE_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  h->launches += (h->launches - before) * (times - 1);  // every replay runs every captured node
  for (int i = 0; i < times; ++i) {
    e = cudaGraphLaunch(gg.e, st);
    if (e != cudaSuccess) return h->fail(DEBYE_ECUDA, "graph launch: %s", cudaGetErrorString(e));
  }
  return DEBYE_OK;
}

int fit_impl(debye_handle h, const debye_spectra* sp, const debye_search* se, int32_t n_max,
             double* eps_inf, double* d_eps, double* tau, double* final_cost, cudaStream_t st,
             const int64_t* rng_id, bool reset_evals) {
  int rc;
  Plan pl;
  if ((rc = h->load_plan(sp, pl, st))) return rc;
  if (pl.nmax_seen > n_max) return h->fail(DEBYE_EINVAL, "n_max = %d < largest N = %d", n_max, pl.nmax_seen);
  if (pl.S == 0) return DEBYE_OK;
  const int P = se->P;
  const int64_t Q = pl.S * (int64_t)P;
  if (Q > ((int64_t)1 << 31) - 1) return h->fail(DEBYE_EINVAL, "S*P exceeds 2^31-1");
  if ((rc = h->prep_spectra(sp, pl, st))) return rc;
  if ((rc = h->build_tables(sp, pl, st))) return rc;   // once per fit: the samples do not change
  int cb, ks;
  choose_layout(P, Q, h->sms, h->forced(), h->tuned, &cb, &ks);
  const bool mixed = h->mixed();
  const int nmax = n_max;

  // ---- swarm state and evaluation plan
  std::vector<int32_t> qb(pl.S), qe(pl.S);
  for (int64_t s = 0; s < pl.S; ++s) {
    qb[s] = (int32_t)(s * P);
    qe[s] = (int32_t)((s + 1) * P);
  }
  UnitGroups g;
  build_units(pl, qb, qe, cb, g);
  if ((rc = h->upload_units(g, h->ws_units, st))) return rc;
  EvalArgs ea{};
  if ((rc = h->ensure_scratch(Q, nmax, h->sb_eval, ea.sc))) return rc;
  SwarmArgs sa{};
  void* p;
  sa.S = pl.S;
  sa.P = P;
  sa.nmax = nmax;
  sa.iters = se->iters;
  sa.seed = se->seed;
  sa.omega = h->opt.pso_omega;
  sa.phi_p = h->opt.pso_phi_p;
  sa.phi_g = h->opt.pso_phi_g;
  sa.de_f_lo = h->opt.de_f_lo;
  sa.de_f_hi = h->opt.de_f_hi;
  sa.de_cr = h->opt.de_cr;
  sa.de_strategy = h->opt.de_strategy;
  sa.da_t0 = h->opt.da_t0;
  sa.da_qa = h->opt.da_qa;
  const bool evolve = se->method == DEBYE_SEARCH_DE;
  const bool anneal = se->method == DEBYE_SEARCH_DA;
  sa.n_poles = sp->n_poles;
  sa.lo = sp->lo;
  sa.hi = sp->hi;
  sa.offsets = sp->offsets;
  sa.rng_id = rng_id;
  const size_t qn = sizeof(double) * (size_t)Q * nmax;
  if ((rc = h->named("swarm.x", qn, &p))) return rc;
  sa.x = (double*)p;
  if ((rc = h->named("swarm.v", qn, &p))) return rc;
  sa.v = (double*)p;
  if ((rc = h->named("swarm.pbx", qn, &p))) return rc;
  sa.pbx = (double*)p;
  if ((rc = h->named("swarm.pbc", sizeof(double) * Q, &p))) return rc;
  sa.pbc = (double*)p;
  if ((rc = h->named("swarm.cost", sizeof(double) * Q, &p))) return rc;
  double* cost = (double*)p;
  if ((rc = h->named("swarm.gbest", sizeof(int32_t) * pl.S, &p))) return rc;
  sa.gbest = (int32_t*)p;
  if ((rc = h->named("swarm.gen", sizeof(int), &p))) return rc;
  sa.gen = (int*)p;
  if (anneal) {
    if ((rc = h->named("anneal.cx", qn, &p))) return rc;
    sa.cx = (double*)p;
    if ((rc = h->named("anneal.ce", sizeof(double) * Q, &p))) return rc;
    sa.ce = (double*)p;
    if ((rc = h->named("anneal.active", Q, &p))) return rc;
    sa.active = (uint8_t*)p;
  }
  sa.trace = se->trace;
  sa.evals = se->evals;
  if (se->evals && reset_evals) cudaMemsetAsync(se->evals, 0, sizeof(double), st);
  cudaMemsetAsync(sa.gen, 0, sizeof(int), st);

  ea.units = (const Unit*)h->ws_units.p;
  ea.theta = sa.x;
  ea.kf32 = (const float4*)h->ws_kf32.p;
  ea.kff = (const float4*)h->ws_kff.p;
  ea.kq32 = ea.kf32 + pl.n_samples;
  ea.kqff = ea.kff + pl.n_samples;
  ea.omega = sp->omega;
  ea.eps_re = sp->eps_re;
  ea.eps_im = sp->eps_im;
  ea.h0 = (const double*)h->ws_h0.p;
  ea.bb = ea.h0 + pl.S;
  ea.lam = h->opt.lam_search;
  ea.ks = ks;
  ea.status = h->d_status;
  ea.n_failed = se->n_failed;
  const int steps = h->opt.refine_steps;

  // generation 0: initial positions (the same for both methods), evaluation, bests
  launch_pso_init(sa, h->sms, st); ++h->launches;
  if ((rc = h->run_eval(ea, g, mixed, steps, cost, nullptr, nullptr, h->sb_eval.g1, cb, st))) return rc;
  launch_pso_best(sa, cost, h->sms, st); ++h->launches;
  if (anneal) {
    launch_da_start(sa, h->sms, st);
    ++h->launches;
  }
  launch_gen_advance(sa.gen, st); ++h->launches;
  if ((rc = h->check_launch("swarm start"))) return rc;
  if (anneal) {
    // one outer iteration: 2 nmax moves (moves beyond 2 N_s are masked for spectrum s),
    // each evaluated and accepted or rejected, then the per-spectrum best and trace
    EvalArgs ev = ea;
    ev.active = sa.active;
    rc = repeat(h, se->iters, st, [&]() -> int {
      for (int j = 0; j < 2 * pl.nmax_seen; ++j) {
        launch_da_visit(sa, j, h->sms, st); ++h->launches;
        int r = h->run_eval(ev, g, mixed, steps, cost, nullptr, nullptr, h->sb_eval.g1, cb, st);
        if (r) return r;
        launch_da_accept(sa, cost, j, h->sms, st); ++h->launches;
      }
      launch_da_best(sa, h->sms, st); ++h->launches;
      launch_gen_advance(sa.gen, st); ++h->launches;
      return h->check_launch("annealing iteration");
    });
  } else rc = repeat(h, se->iters, st, [&]() -> int {
    if (evolve) launch_de_trial(sa, h->sms, st);
    else launch_pso_move(sa, h->sms, st);
    ++h->launches;
    int r = h->run_eval(ea, g, mixed, steps, cost, nullptr, nullptr, h->sb_eval.g1, cb, st);
    if (r) return r;
    launch_pso_best(sa, cost, h->sms, st); ++h->launches;
    launch_gen_advance(sa.gen, st); ++h->launches;
    return h->check_launch("generation");
  });
  if (rc) return rc;

  // ---- polish
  PolishArgs pa{};
  const int T = std::min(se->polish_topk, P);
  pa.T = T;
  if (T > 0) {
    pa.L = pl.S * (int64_t)T;
    pa.R = POLISH_R;
    pa.nmax = nmax;
    pa.m = h->opt.lbfgs_m;
    pa.max_trials = h->opt.lbfgs_max_trials;
    pa.c1 = h->opt.lbfgs_c1;
    pa.evals = se->evals;
    const int64_t L = pa.L, QT = L * pa.R;
    const size_t ln = sizeof(double) * (size_t)L * nmax;
    if ((rc = h->named("pol.th", ln, &p))) return rc;
    pa.th = (double*)p;
    if ((rc = h->named("pol.f", sizeof(double) * L, &p))) return rc;
    pa.f = (double*)p;
    if ((rc = h->named("pol.g", ln, &p))) return rc;
    pa.g = (double*)p;
    if ((rc = h->named("pol.dir", ln, &p))) return rc;
    pa.dir = (double*)p;
    if ((rc = h->named("pol.hs", ln * pa.m, &p))) return rc;
    pa.hs = (double*)p;
    if ((rc = h->named("pol.hy", ln * pa.m, &p))) return rc;
    pa.hy = (double*)p;
    if ((rc = h->named("pol.int", sizeof(int32_t) * 4 * L, &p))) return rc;
    pa.hcount = (int32_t*)p;
    pa.t0 = pa.hcount + L;
    pa.done = pa.hcount + 2 * L;
    pa.acc = pa.hcount + 3 * L;
    if ((rc = h->named("pol.tth", sizeof(double) * QT * nmax, &p))) return rc;
    pa.tth = (double*)p;
    if ((rc = h->named("pol.tcost", sizeof(double) * QT, &p))) return rc;
    pa.tcost = (double*)p;
    if ((rc = h->named("pol.active", QT, &p))) return rc;
    pa.active = (uint8_t*)p;
    if ((rc = h->named("pol.ath", ln, &p))) return rc;
    pa.ath = (double*)p;
    if ((rc = h->named("pol.acost", sizeof(double) * L, &p))) return rc;
    pa.acost = (double*)p;
    if ((rc = h->named("pol.agrad", ln, &p))) return rc;
    pa.agrad = (double*)p;
    if ((rc = h->named("pol.aactive", L, &p))) return rc;
    pa.aactive = (uint8_t*)p;

    // trial steps: candidate l * R + t; accepted points: candidate l
    std::vector<int32_t> pb(pl.S), pe(pl.S), ab(pl.S), ae(pl.S);
    for (int64_t s = 0; s < pl.S; ++s) {
      pb[s] = (int32_t)(s * T * pa.R);
      pe[s] = (int32_t)((s + 1) * T * pa.R);
      ab[s] = (int32_t)(s * T);
      ae[s] = (int32_t)((s + 1) * T);
    }
    // trial steps: one work unit per line (its R step lengths), so that a unit whose line
    // has stopped searching exits at once and an active one has no idle candidates
    int cba, ksa;
    const int cbp = pa.R, ksp = MAX_BLOCK / pa.R;
    if (h->tuned_polish.cb > 0) {   // debye_autotune's choice for this shape
      cba = h->tuned_polish.cb;
      ksa = h->tuned_polish.ks;
    } else {
      choose_layout(T, pl.S * T, h->sms, h->forced(), h->tuned, &cba, &ksa);
    }
    UnitGroups gp, ga;
    build_units(pl, pb, pe, cbp, gp);
    build_units(pl, ab, ae, cba, ga);
    if ((rc = h->upload_units(gp, h->named_bufs["pol.units"], st))) return rc;
    if ((rc = h->upload_units(ga, h->named_bufs["pol.aunits"], st))) return rc;
    EvalArgs ep = ea;
    if ((rc = h->ensure_scratch(QT, nmax, h->sb_polish, ep.sc))) return rc;
    ep.units = (const Unit*)h->named_bufs["pol.units"].p;
    ep.theta = pa.tth;
    ep.active = pa.active;
    ep.ks = ksp;
    EvalArgs eg = ea;
    if ((rc = h->ensure_scratch(L, nmax, h->sb_polish_acc, eg.sc))) return rc;
    eg.units = (const Unit*)h->named_bufs["pol.aunits"].p;
    eg.theta = pa.ath;
    eg.active = pa.aactive;
    eg.ks = ksa;

    launch_topk(sa, pa, h->sms, st); ++h->launches;
    launch_polish_start(pa, h->sms, st); ++h->launches;
    if ((rc = h->run_eval(eg, ga, mixed, h->eval_steps(true), pa.acost, nullptr, pa.agrad, h->sb_polish_acc.g1,
                          cba, st)))
      return rc;
    launch_polish_take0(pa, h->sms, st); ++h->launches;
    if (se->evals) {  // the start evaluation of every line
      double add = 0.0;
      for (int64_t s = 0; s < pl.S; ++s) add += (double)T * (double)(pl.offs[s + 1] - pl.offs[s]);
      launch_add_scalar(se->evals, add, st); ++h->launches;
    }
    if ((rc = h->check_launch("polish start"))) return rc;
    const int rounds = (pa.max_trials - 1 + pa.R - 1) / pa.R;
    rc = repeat(h, se->polish_iters, st, [&]() -> int {
      launch_polish_dir(pa, sp->n_poles, sp->lo, sp->hi, h->sms, st); ++h->launches;
      // the full step of every line, with its gradient (most lines accept it)
      int e = h->run_eval(eg, ga, mixed, h->eval_steps(true), pa.acost, nullptr, pa.agrad, h->sb_polish_acc.g1,
                          cba, st);
      if (e) return e;
      launch_polish_first(pa, sp->n_poles, sp->lo, sp->hi, sp->offsets, h->sms, st); ++h->launches;
      for (int r = 0; r < rounds; ++r) {
        // Armijo needs only costs: the backtracking steps are evaluated without gradients
        e = h->run_eval(ep, gp, mixed, h->eval_steps(false), pa.tcost, nullptr, nullptr, h->sb_polish.g1, cbp, st);
        if (e) return e;
        launch_polish_accept(pa, sp->n_poles, sp->lo, sp->hi, sp->offsets, h->sms, st); ++h->launches;
      }
      // cost and gradient at the points accepted by backtracking, then the L-BFGS update
      e = h->run_eval(eg, ga, mixed, h->eval_steps(true), pa.acost, nullptr, pa.agrad, h->sb_polish_acc.g1, cba,
                      st);
      if (e) return e;
      launch_polish_take(pa, sp->n_poles, h->sms, st); ++h->launches;
      return h->check_launch("polish iteration");
    });
    if (rc) return rc;
  }

  // ---- final FP64 re-solve at lam_final, sorted result
  const int64_t S = pl.S;
  if ((rc = h->named("fin.theta", sizeof(double) * S * nmax, &p))) return rc;
  double* th_best = (double*)p;
  if ((rc = h->named("fin.w", sizeof(double) * S * (nmax + 1), &p))) return rc;
  double* w_best = (double*)p;
  if ((rc = h->named("fin.cost", sizeof(double) * S, &p))) return rc;
  double* c_best = (double*)p;
  launch_pick_best(sa, pa, th_best, h->sms, st); ++h->launches;
  std::vector<int32_t> fb(S), fe(S);
  for (int64_t s = 0; s < S; ++s) {
    fb[s] = (int32_t)s;
    fe[s] = (int32_t)(s + 1);
  }
  int cbf, ksf;
  choose_layout(1, S, h->sms, Layout{}, Layout{}, &cbf, &ksf);
  UnitGroups gf;
  build_units(pl, fb, fe, cbf, gf);
  if ((rc = h->upload_units(gf, h->named_bufs["fin.units"], st))) return rc;
  EvalArgs ef = ea;
  if ((rc = h->ensure_scratch(S, nmax, h->sb_final, ef.sc))) return rc;
  ef.units = (const Unit*)h->named_bufs["fin.units"].p;
  ef.theta = th_best;
  ef.active = nullptr;
  ef.ks = ksf;
  ef.lam = h->opt.lam_final;
  if ((rc = h->run_eval(ef, gf, false, 2, c_best, w_best, nullptr, h->sb_final.g1, cbf, st))) return rc;
  launch_assemble(S, nmax, sp->n_poles, th_best, w_best, c_best, eps_inf, d_eps, tau, final_cost, h->sms, st);
  ++h->launches;
  return h->check_launch("assemble");
}

extern "C" int debye_fit_batch(debye_handle h, const debye_spectra* sp, const debye_search* se,
                               int32_t n_max, double* eps_inf, double* d_eps, double* tau,
                               double* final_cost, cudaStream_t st) {
  if (!h) return DEBYE_EINVAL;
  h->err.clear();
  if (!sp || !se) return h->fail(DEBYE_EINVAL, "spectra or search is NULL");
  if (se->P < 1 || se->P > 32768) return h->fail(DEBYE_EINVAL, "P = %d outside 1..32768", se->P);
  if (se->iters < 0) return h->fail(DEBYE_EINVAL, "iters < 0");
  if (se->method != DEBYE_SEARCH_PSO && se->method != DEBYE_SEARCH_DE && se->method != DEBYE_SEARCH_DA)
    return h->fail(DEBYE_EINVAL, "method must be DEBYE_SEARCH_PSO, DEBYE_SEARCH_DE or DEBYE_SEARCH_DA");
  if (se->method == DEBYE_SEARCH_DA && se->iters > 1000)
    return h->fail(DEBYE_EINVAL, "dual annealing: at most 1000 outer iterations");
  if (se->method == DEBYE_SEARCH_DE && se->iters > 0 &&
      se->P < (h->opt.de_strategy == DEBYE_DE_RAND1 ? 4 : 3))
    return h->fail(DEBYE_EINVAL, "differential evolution needs P >= %d",
                   h->opt.de_strategy == DEBYE_DE_RAND1 ? 4 : 3);
  if (se->polish_topk < 0 || se->polish_topk > 64) return h->fail(DEBYE_EINVAL, "polish_topk outside 0..64");
  if (se->polish_iters < 0) return h->fail(DEBYE_EINVAL, "polish_iters < 0");
  if (n_max < 1 || n_max > NMAX) return h->fail(DEBYE_EINVAL, "n_max = %d outside 1..%d", n_max, NMAX);
  if (sp->S > 0 && (!eps_inf || !d_eps || !tau || !final_cost)) return h->fail(DEBYE_EINVAL, "an output is NULL");
  cudaStream_t ws = h->work_stream;
  cudaEventRecord(h->ev_in, st);
  cudaStreamWaitEvent(ws, h->ev_in, 0);
  int rc = fit_impl(h, sp, se, n_max, eps_inf, d_eps, tau, final_cost, ws, nullptr, true);
  cudaEventRecord(h->ev_out, ws);
  cudaStreamWaitEvent(st, h->ev_out, 0);
  return rc;
}
