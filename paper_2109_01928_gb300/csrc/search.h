// Device-side state of the particle swarm and the L-BFGS polish.
#pragma once
#include "common.cuh"

namespace debyefit {

struct SwarmArgs {
  int64_t S;
  int32_t P, nmax, iters;
  uint64_t seed;
  double omega, phi_p, phi_g;
  double de_f_lo, de_f_hi, de_cr;  // differential evolution coefficients
  int32_t de_strategy;             // DEBYE_DE_RAND1 or DEBYE_DE_BEST1
  double da_t0, da_qa;             // dual annealing: initial temperature, acceptance parameter
  const int32_t* n_poles;
  const double* lo;
  const double* hi;
  const int64_t* offsets;
  const int64_t* rng_id;  // [S] spectrum index used in the generator's keys, or nullptr (= s)
  double* x;       // [S*P][nmax] positions (log10 tau); differential evolution: trial vectors
  double* v;       // [S*P][nmax] velocities (swarm only)
  double* pbx;     // [S*P][nmax] personal-best positions; differential evolution: the population
  double* pbc;     // [S*P]       personal-best costs; differential evolution: population costs
  int32_t* gbest;  // [S]         global-best particle
  double* cx;      // [S*P][nmax] dual annealing: current chain states
  double* ce;      // [S*P]       dual annealing: current energies
  uint8_t* active; // [S*P]       dual annealing: member moved in this step (evaluation mask)
  int* gen;        // generation counter (device)
  double* trace;   // [S][iters+1] or nullptr
  double* evals;   // [1] or nullptr
};

struct PolishArgs {
  int64_t L;       // lines = S * T
  int32_t T;       // lines per spectrum
  int32_t R;       // trial step lengths per backtracking round (after the full step)
  int32_t nmax, m, max_trials;
  double c1;
  double* th;      // [L][nmax] current point
  double* f;       // [L]
  double* g;       // [L][nmax]
  double* dir;     // [L][nmax]
  double* hs;      // [L][m][nmax] history s (oldest first)
  double* hy;      // [L][m][nmax] history y
  int32_t* hcount; // [L]
  int32_t* t0;     // [L] first trial index of the next backtracking round
  int32_t* done;   // [L] line finished (no acceptable step or non-finite)
  int32_t* acc;    // [L] step accepted in this iteration (acost, agrad at ath ready after the last evaluation)
  double* tth;     // [L*R][nmax] trial points
  double* tcost;   // [L*R]
  uint8_t* active; // [L*R] trial needs evaluation
  // the accepted point of each line, evaluated with its gradient
  double* ath;     // [L][nmax] accepted point
  double* acost;   // [L]
  double* agrad;   // [L][nmax]
  uint8_t* aactive;// [L] ath needs a cost + gradient evaluation (the full step, or a later accepted trial)
  double* evals;   // [1] or nullptr
};

void launch_pso_init(const SwarmArgs& a, int sms, cudaStream_t st);
void launch_pso_move(const SwarmArgs& a, int sms, cudaStream_t st);
void launch_de_trial(const SwarmArgs& a, int sms, cudaStream_t st);
void launch_da_start(const SwarmArgs& a, int sms, cudaStream_t st);
void launch_da_visit(const SwarmArgs& a, int j, int sms, cudaStream_t st);
void launch_da_accept(const SwarmArgs& a, const double* cost, int j, int sms, cudaStream_t st);
void launch_da_best(const SwarmArgs& a, int sms, cudaStream_t st);
void launch_pso_best(const SwarmArgs& a, const double* cost, int sms, cudaStream_t st);
void launch_gen_advance(int* gen, cudaStream_t st);
void launch_add_scalar(double* dst, double v, cudaStream_t st);
void launch_topk(const SwarmArgs& a, const PolishArgs& pa, int sms, cudaStream_t st);
void launch_polish_start(const PolishArgs& pa, int sms, cudaStream_t st);
void launch_polish_take0(const PolishArgs& pa, int sms, cudaStream_t st);
void launch_polish_dir(const PolishArgs& pa, const int32_t* n_poles, const double* lo, const double* hi,
                       int sms, cudaStream_t st);
void launch_polish_first(const PolishArgs& pa, const int32_t* n_poles, const double* lo, const double* hi,
                         const int64_t* offsets, int sms, cudaStream_t st);
void launch_polish_accept(const PolishArgs& pa, const int32_t* n_poles, const double* lo, const double* hi,
                          const int64_t* offsets, int sms, cudaStream_t st);
void launch_polish_take(const PolishArgs& pa, const int32_t* n_poles, int sms, cudaStream_t st);
void launch_pick_best(const SwarmArgs& a, const PolishArgs& pa, double* out_theta, int sms, cudaStream_t st);
void launch_assemble(int64_t S, int nmax, const int32_t* n_poles, const double* theta, const double* weights,
                     const double* cost, double* eps_inf, double* d_eps, double* tau, double* final_cost,
                     int sms, cudaStream_t st);

}  // namespace debyefit
