// Allocation-free population evaluation (debye_eval_population_noalloc).
//
// Some callers cannot let this library allocate device memory: an application
// that embeds the fitter (for example an FDTD solver that owns a fixed device
// memory budget and pre-allocates everything up front), or a latency-critical
// loop in which cudaMalloc/cudaFree, which may synchronise the device, are not
// acceptable. The handle-based entry points allocate their workspaces on first
// use; this one instead uses a fixed scratch array that lives in the library's
// own device image, so a call allocates nothing. The caller still provides the
// inputs and the outputs.
//
// The scratch is one file-scope array per device, held from the time the
// library's device code is loaded on that device until the process exits.
// Every call on a device uses the same array and leaves its contents behind;
// calls whose work overlaps on the GPU (different streams or host threads,
// without ordering between them) race on it and give wrong results.
#include <cuda.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "launch.h"

namespace debyefit {
namespace {

constexpr size_t SCRATCH_BYTES = DEBYE_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_UNITS = 4096;
constexpr int MAX_DEVICES = 64;
// every sample takes 64 B of the scratch (two float4 records in kf32 and in kff)
constexpr int64_t MAX_SAMPLES = (int64_t)(SCRATCH_BYTES / (4 * sizeof(float4)));

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch per device. In host code `g_scratch` names a host
// stand-in, not device memory, so the address must come from the runtime
// (cudaGetSymbolAddress, with the device current). The address is looked up
// once per device and context: a cudaDeviceReset destroys the device's context
// and the next context may load the library's device image elsewhere, so a
// cached address is reused only while the context that it was looked up in
// (identified by the driver's unique context id) is still current. Where the
// context id cannot be queried, every call looks the address up.
struct ScratchSlot {
  void* ptr = nullptr;
  unsigned long long ctx_id = 0;
  bool valid = false;
};
std::mutex g_mu;
ScratchSlot g_slot[MAX_DEVICES];

typedef CUresult(CUDAAPI* ctx_get_current_fn)(CUcontext*);
typedef CUresult(CUDAAPI* ctx_get_id_fn)(CUcontext, unsigned long long*);
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;
bool g_entry_points_looked_up = false;

// Driver entry points for the context id (no link-time dependency on libcuda).
void lookup_entry_points() {
  if (g_entry_points_looked_up) return;
  g_entry_points_looked_up = true;
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_current = (ctx_get_current_fn)f;
  f = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_ctx_get_id = (ctx_get_id_fn)f;
  cudaGetLastError();
}

// Unique id of the current context; false if there is none or it cannot be queried.
bool current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) return false;
  CUcontext c = nullptr;
  if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return false;
  return g_ctx_get_id(c, id) == CUDA_SUCCESS;
}

int scratch_address(void** out, char* err, int err_len) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    if (err && err_len > 0) snprintf(err, err_len, "no usable CUDA device");
    return DEBYE_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  lookup_entry_points();
  unsigned long long id = 0;
  ScratchSlot& slot = g_slot[dev];
  if (slot.valid && current_context_id(&id) && id == slot.ctx_id) {
    *out = slot.ptr;
    return DEBYE_OK;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    if (err && err_len > 0)
      snprintf(err, err_len, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
    return DEBYE_ECUDA;
  }
  slot.ptr = p;
  slot.valid = current_context_id(&id);   // the lookup made the device's context current
  slot.ctx_id = id;
  *out = p;
  return DEBYE_OK;
}

// Bump allocator over the fixed array (offsets only, nothing is allocated).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  bool ok = true;
  void* take(size_t bytes) {
    const size_t off = (used + 255) & ~(size_t)255;
    if (!ok || off > SCRATCH_BYTES || bytes > SCRATCH_BYTES - off) {
      ok = false;
      return nullptr;
    }
    used = off + bytes;
    return base + off;
  }
};

int fail_msg(int code, char* err, int err_len, const char* msg) {
  if (err && err_len > 0) snprintf(err, err_len, "%s", msg);
  return code;
}

}  // namespace
}  // namespace debyefit

using namespace debyefit;

extern "C" int debye_eval_population_noalloc(const debye_options* opt_in, const debye_spectra* sp,
                                             int32_t P, int32_t n_max, const double* theta,
                                             double* cost, double* weights, char* err,
                                             int32_t err_len, cudaStream_t st) {
  if (err && err_len > 0) err[0] = '\0';
  debye_options opt;
  if (opt_in) opt = *opt_in;
  else debye_default_options(&opt);
  if (opt.precision != DEBYE_PREC_FP64 && opt.precision != DEBYE_PREC_MIXED && opt.precision != DEBYE_PREC_FP64_SUMS &&
      opt.precision != DEBYE_PREC_MIXED_TABLE)
    return fail_msg(DEBYE_EINVAL, err, err_len, "precision must be DEBYE_PREC_FP64, _MIXED, _FP64_SUMS or _MIXED_TABLE");
  if (opt.refine_steps < 1 || opt.refine_steps > 4 || !(opt.lam_search >= 0.0))
    return fail_msg(DEBYE_EINVAL, err, err_len, "refine_steps outside 1..4 or negative lam_search");
  if (!sp) return fail_msg(DEBYE_EINVAL, err, err_len, "spectra is NULL");
  if (sp->S < 0 || P < 1 || n_max < 1 || n_max > NMAX)
    return fail_msg(DEBYE_EINVAL, err, err_len, "S < 0, P < 1 or n_max outside 1..DEBYE_MAX_POLES");
  if (sp->S == 0) return DEBYE_OK;
  if (!sp->offsets_host || !sp->n_poles_host)
    return fail_msg(DEBYE_EINVAL, err, err_len, "offsets_host and n_poles_host are required");
  if (!sp->offsets || !sp->omega || !sp->eps_re || !sp->eps_im || !sp->n_poles || !sp->lo || !sp->hi ||
      !theta || !cost)
    return fail_msg(DEBYE_EINVAL, err, err_len, "a required pointer is NULL");
  const int64_t S = sp->S;
  const int64_t Q = S * (int64_t)P;
  if (Q > ((int64_t)1 << 31) - 1) return fail_msg(DEBYE_EINVAL, err, err_len, "S*P exceeds 2^31-1");
  // Bounds that keep every byte count below the scratch size (no size_t overflow in
  // the carving below): 8 B per candidate and 16 B per spectrum at the very least.
  if (Q > (int64_t)(SCRATCH_BYTES / sizeof(double)) || S > (int64_t)(SCRATCH_BYTES / (2 * sizeof(double))))
    return fail_msg(DEBYE_EINVAL, err, err_len, "batch needs more than the allocation-free scratch");
  if (opt.lanes_per_candidate != 0 && (opt.lanes_per_candidate < 1 || opt.lanes_per_candidate > 32 ||
                                       (opt.lanes_per_candidate & (opt.lanes_per_candidate - 1))))
    return fail_msg(DEBYE_EINVAL, err, err_len, "lanes_per_candidate");
  {
    const int blk = opt.cands_per_block * std::max(opt.lanes_per_candidate, 1);
    if (opt.cands_per_block < 0 || (opt.cands_per_block && (blk > MAX_BLOCK || blk % 32)))
      return fail_msg(DEBYE_EINVAL, err, err_len,
                      "cands_per_block x lanes_per_candidate must be a multiple of 32, at most 128");
  }
  int cb, ks;
  int sms_l = 1, dev_l = 0;
  cudaGetDevice(&dev_l);
  cudaDeviceGetAttribute(&sms_l, cudaDevAttrMultiProcessorCount, dev_l);
  // one lane per candidate for populations of a warp or more (as large batches get), so
  // the number of work units stays small
  choose_layout(P, (int64_t)1 << 40, sms_l, Layout{opt.cands_per_block, opt.lanes_per_candidate}, Layout{}, &cb,
                &ks);
  const int64_t* offs = sp->offsets_host;
  if (offs[0] != 0) return fail_msg(DEBYE_EINVAL, err, err_len, "offsets[0] must be 0");

  // work units, grouped by pole bucket, on the host stack
  Unit units[MAX_UNITS];
  int begin[N_BUCKETS + 1];
  int n_units = 0;
  for (int b = 0; b < N_BUCKETS; ++b) {
    begin[b] = n_units;
    for (int64_t s = 0; s < S; ++s) {
      const int N = sp->n_poles_host[s];
      if (N < 1 || N > n_max || offs[s + 1] < offs[s])
        return fail_msg(DEBYE_EINVAL, err, err_len, "n_poles outside 1..n_max or offsets decreasing");
      if (offs[s + 1] > MAX_SAMPLES)
        return fail_msg(DEBYE_EINVAL, err, err_len, "batch has more frequency samples than the "
                        "allocation-free scratch holds (64 B per sample)");
      if (bucket_of(N) != b) continue;
      for (int64_t q = s * P; q < (s + 1) * P; q += cb) {
        if (n_units == MAX_UNITS)
          return fail_msg(DEBYE_EINVAL, err, err_len, "batch needs more than 4096 work units");
        Unit& u = units[n_units++];
        u.s = (int32_t)s;
        u.q0 = (int32_t)q;
        u.q1 = (int32_t)std::min<int64_t>((s + 1) * P, q + cb);
        u.N = N;
        u.k0 = offs[s];
        u.k1 = offs[s + 1];
      }
    }
  }
  begin[N_BUCKETS] = n_units;
  const int64_t n_samples = offs[S];

  // carve the fixed scratch: status, units, per-sample, per-spectrum and per-candidate arrays
  void* base = nullptr;
  int rc = scratch_address(&base, err, err_len);
  if (rc) return rc;
  Carve cv{(unsigned char*)base};
  const int nm1 = n_max + 1;
  const int npk = nm1 * (nm1 + 1) / 2;
  int* status = (int*)cv.take(sizeof(int));
  Unit* d_units = (Unit*)cv.take(sizeof(Unit) * n_units);
  float4* kf32 = (float4*)cv.take(sizeof(float4) * 2 * n_samples);
  float4* kff = (float4*)cv.take(sizeof(float4) * 2 * n_samples);
  double* h0 = (double*)cv.take(sizeof(double) * 2 * S);   // sum eps', then b^T b
  Scratch sc{};
  sc.Q = Q;
  sc.nmax = n_max;
  sc.ng = npk + nm1;
  sc.G = (double*)cv.take(sizeof(double) * sc.ng * Q);
  sc.L = (double*)cv.take(sizeof(double) * npk * Q);
  sc.dinv = (double*)cv.take(sizeof(double) * nm1 * Q);
  sc.x = (double*)cv.take(sizeof(double) * nm1 * Q);
  sc.xh = (double*)cv.take(sizeof(double) * nm1 * Q);
  sc.w = (double*)cv.take(sizeof(double) * nm1 * Q);
  double* g1 = (double*)cv.take(sizeof(double) * nm1 * Q);
  sc.rt = (double*)cv.take(sizeof(double) * (nm1 + 1) * Q);
  sc.gt = sc.G;
  sc.fail = (int32_t*)cv.take(sizeof(int32_t) * Q);
  if (!cv.ok) {
    if (err && err_len > 0)
      snprintf(err, err_len, "batch needs more than the %zu-byte allocation-free scratch "
               "(S=%lld, P=%d, n_max=%d, samples=%lld)", SCRATCH_BYTES, (long long)S, P, n_max,
               (long long)n_samples);
    return DEBYE_EINVAL;
  }

  int sms = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_units, units, sizeof(Unit) * n_units, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail_msg(DEBYE_ECUDA, err, err_len, cudaGetErrorString(e));
  }
  launch_prep(n_samples, S, sp->offsets, sp->omega, sp->eps_re, sp->eps_im, sp->lo, sp->hi, kf32, kff, h0,
              status, sms, st);

  EvalArgs a{};
  a.units = d_units;
  a.n_units = n_units;
  a.theta = theta;
  a.kf32 = kf32;
  a.kff = kff;
  a.kq32 = kf32 + n_samples;
  a.kqff = kff + n_samples;
  a.omega = sp->omega;
  a.eps_re = sp->eps_re;
  a.eps_im = sp->eps_im;
  a.h0 = h0;
  a.bb = h0 + S;
  a.active = nullptr;
  a.ks = ks;
  a.lam = opt.lam_search;
  a.sc = sc;
  a.status = status;
  const bool mixed = opt.precision == DEBYE_PREC_MIXED || opt.precision == DEBYE_PREC_MIXED_TABLE;   // direct sums
  auto per_bucket = [&](int phase) {
    for (int b = 0; b < N_BUCKETS; ++b) {
      const int n = begin[b + 1] - begin[b];
      if (!n) continue;
      EvalArgs ab = a;
      ab.units = a.units + begin[b];
      ab.n_units = n;
      const int grid = std::max(1, std::min(n, sms * 16));
      launch_pass(b + 1, phase, ab, grid, cb * ks, st);
    }
  };
  if (mixed) {
    // one float-float column-sum pass, weights and cost from the exact Gram identity
    per_bucket(PH_SUMS);
    launch_solve_sums(a, cost, weights, nullptr, warp_round(cb), sms, st);
  } else {
    per_bucket(opt.precision == DEBYE_PREC_FP64_SUMS ? PH_GRAM_SUMS : PH_GRAM);
    launch_solve(a, warp_round(cb), sms, st);
    for (int it = 0; it < opt.refine_steps; ++it) {
      per_bucket(PH_REFINE);
      launch_finish(a, it + 1 == opt.refine_steps ? 1 : 0, cost, weights, g1, warp_round(cb), sms, st);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_msg(DEBYE_ECUDA, err, err_len, cudaGetErrorString(e));

  // wait for the work and report what the device detected (non-finite input, bounds)
  int dstatus = 0;
  e = cudaMemcpyAsync(&dstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_msg(DEBYE_ECUDA, err, err_len, cudaGetErrorString(e));
  if (dstatus != 0) return fail_msg(dstatus, err, err_len, "device reported invalid input (non-finite or bounds)");
  return DEBYE_OK;
}
