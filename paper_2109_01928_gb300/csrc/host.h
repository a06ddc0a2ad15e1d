// Host-side state of a libdebyefit handle.
#pragma once
#include <cstdint>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "launch.h"

namespace debyefit {

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

// Host view of a ragged batch: sample offsets and pole counts.
struct Plan {
  int64_t S = 0;
  int64_t n_samples = 0;
  int32_t nmax_seen = 0;
  std::vector<int64_t> offs;
  std::vector<int32_t> npol;
};

// Work units grouped by pole bucket: bucket b owns units[begin[b] .. begin[b+1]).
struct UnitGroups {
  std::vector<Unit> units;
  int begin[N_BUCKETS + 1] = {0};
};

struct ScratchBufs {
  Buf G, L, vec, rt, fail;
  double* g1 = nullptr;
};

void build_units(const Plan& pl, const std::vector<int32_t>& qb, const std::vector<int32_t>& qe,
                 int cb, UnitGroups& g);

}  // namespace debyefit

// Whole fit of a batch on stream st (the body of debye_fit_batch). rng_id [S]
// (device, or nullptr) replaces the batch index in the generator's keys;
// reset_evals zeroes se->evals first.
int fit_impl(struct debye_ctx* h, const debye_spectra* sp, const debye_search* se, int32_t n_max,
             double* eps_inf, double* d_eps, double* tau, double* final_cost, cudaStream_t st,
             const int64_t* rng_id, bool reset_evals);

namespace debyefit {

}  // namespace debyefit

struct debye_ctx {
  debye_options opt{};
  int device = 0;
  int sms = 1;
  int* d_status = nullptr;
  std::string err;
  cudaStream_t capturing_stream = nullptr;
  // Test hook: return true to make the next workspace allocation fail.
  std::function<bool(size_t)> alloc_hook;

  cudaStream_t work_stream = nullptr;  // non-blocking stream of debye_fit_batch
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // Pole buckets of one pass run concurrently: bucket b > first on side[b], forked
  // from and joined back to the launching stream (so their tails overlap).
  cudaStream_t side[debyefit::N_BUCKETS] = {nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[debyefit::N_BUCKETS] = {nullptr};

  debyefit::Buf ws_kf32, ws_kff, ws_h0, ws_units;
  debyefit::Buf ws_tab_units;    // units of the column-sum tables' node pass
  debyefit::TabView tab{};       // column-sum tables of the current call (DEBYE_PREC_MIXED_TABLE)
  debyefit::ScratchBufs sb_eval, sb_polish, sb_polish_acc, sb_final;
  std::map<std::string, debyefit::Buf> named_bufs;  // swarm / polish / result state

  // kernel timing (debye_profile_*)
  struct ProfEntry {
    int kind;
    double flops;
    cudaEvent_t a, b;
  };
  int64_t launches = 0;  // kernel launches enqueued (graph replays count every node)
  debyefit::Layout tuned;         // full-population layout chosen by debye_autotune (unset: not tuned)
  debyefit::Layout tuned_polish;  // layout of the polish's accepted points (debye_autotune)
  debyefit::Layout forced() const { return debyefit::Layout{opt.cands_per_block, opt.lanes_per_candidate}; }
  bool prof_on = false;
  std::vector<ProfEntry> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  int64_t prof_launches[DEBYE_KERNEL_KINDS] = {0};
  double prof_ms[DEBYE_KERNEL_KINDS] = {0};
  double prof_flops[DEBYE_KERNEL_KINDS] = {0};
  cudaEvent_t prof_event();
  void prof_begin(int kind, double flops, cudaStream_t st, ProfEntry& e);
  void prof_end(ProfEntry& e, cudaStream_t st);
  int prof_collect();

  int fail(int code, const char* fmt, ...);
  int ensure(debyefit::Buf& b, size_t bytes, const char* what);
  int check_launch(const char* what);
  int load_plan(const debye_spectra* sp, debyefit::Plan& pl, cudaStream_t st);
  int prep_spectra(const debye_spectra* sp, const debyefit::Plan& pl, cudaStream_t st);
  int upload_units(const debyefit::UnitGroups& g, debyefit::Buf& dst, cudaStream_t st);
  int ensure_scratch(int64_t Q, int nmax, debyefit::ScratchBufs& sb, debyefit::Scratch& sc);
  int run_eval(debyefit::EvalArgs a, const debyefit::UnitGroups& g, bool mixed, int steps,
               double* cost, double* weights, double* grad, double* g1, int cb, cudaStream_t st);
  int eval_steps(bool with_grad) const;
  // Mixed precision: column sums and the Gram identity (direct or tabulated sums).
  bool mixed() const { return opt.precision == DEBYE_PREC_MIXED || opt.precision == DEBYE_PREC_MIXED_TABLE; }
  // DEBYE_PREC_MIXED_TABLE: build every spectrum's column-sum tables (after
  // prep_spectra) and point `tab` at them; a no-op for the other precisions.
  int build_tables(const debye_spectra* sp, const debyefit::Plan& pl, cudaStream_t st);
  int named(const char* name, size_t bytes, void** out);

  void free_buf(debyefit::Buf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
  }
  void release() {
    free_buf(ws_kf32);
    free_buf(ws_kff);
    free_buf(ws_h0);
    free_buf(ws_units);
    free_buf(ws_tab_units);
    for (debyefit::ScratchBufs* sb : {&sb_eval, &sb_polish, &sb_polish_acc, &sb_final}) {
      free_buf(sb->G);
      free_buf(sb->L);
      free_buf(sb->vec);
      free_buf(sb->rt);
      free_buf(sb->fail);
    }
    for (auto& kv : named_bufs) free_buf(kv.second);
    named_bufs.clear();
    if (d_status) cudaFree(d_status);
    d_status = nullptr;
    prof_collect();
    for (cudaEvent_t e : prof_pool) cudaEventDestroy(e);
    prof_pool.clear();
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_fork) cudaEventDestroy(ev_fork);
    ev_fork = nullptr;
    for (int b = 0; b < debyefit::N_BUCKETS; ++b) {
      if (ev_join[b]) cudaEventDestroy(ev_join[b]);
      if (side[b]) cudaStreamDestroy(side[b]);
      ev_join[b] = nullptr;
      side[b] = nullptr;
    }
    if (work_stream) cudaStreamDestroy(work_stream);
    ev_in = ev_out = nullptr;
    work_stream = nullptr;
  }
};
