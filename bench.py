"""Throughput of batched multi-Debye fitting on GB300.

One step = one debye_fit_batch over the whole workload: seeded particle swarm
(every generation evaluates the damped least-squares cost of every particle),
L-BFGS polish of the best personal bests, final FP64 re-solve. The metric is
candidate evaluations x frequency samples per second (cand*K/s), counted on the
device over swarm and polish evaluations. The headline workload is the
1024-spectrum mixed-model batch in mixed precision, next to the plain FP64
evaluator on the same fit; the single-spectrum, differentiation and tabulated
workloads are measured under "configs".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--configs all|none|name,...] [--no-fp64] [--no-cpu-baseline]

With N > 1 (torchrun) every rank fits its own batch of the same shape (seed =
rank): the spectra are independent, so there is no data-path collective, and
the value is the total over ranks divided by the slowest rank's time (weak
scaling). Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "mixed_1024"
# per workload: particles, swarm generations after the first, polished candidates, L-BFGS iterations
SETTINGS = {"mixed_1024": (256, 200, 8, 50), "single_hn_k50": (64, 100, 8, 50),
            "hn_256_k2000": (4096, 0, 32, 50), "tabulated_16384_k4096": (512, 100, 8, 50)}
EXTRA_CONFIGS = ("single_hn_k50", "hn_256_k2000", "tabulated_16384_k4096")
METRIC = "candidate cost evals x K per sec (batched mixed-precision fit)"
UNIT = "cand*K/s"
# ALU peaks from unit counts and the maximum SM clock: FP32, 152 SMs x 128 lanes x 2 FLOP
# per FMA; FP64, the nominal GB300 rate (1.25 TFLOP/s dense, 1/64 of FP32)
SMS, SM_MAX_MHZ = 152, 2070.0
PEAK_FP32 = SMS * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP64 = 1.25
KERNEL_SOURCES = ["paper_2109_01928_gb300/csrc/eval.cuh", "paper_2109_01928_gb300/csrc/common.cuh"]
CTL_REL = 1e-9          # relative perturbation of the damping in the FP64 control fit
TAB_SAMPLE = 64         # spectra of the tabulated workload's oracle sample


def f_alg(N):
    """Algorithmic FP32 FLOPs per cand*K of one cost evaluation by the direct method:
    basis 4N + unique Gram / right-hand-side products 2(N+2)^2 (FMA = 2)."""
    N = np.asarray(N, dtype=np.float64)
    return 4 * N + 2 * (N + 2) ** 2


# ------------------------------------------------------------------ replicas (one process per GPU)

def replica_workload(name: str, rank: int):
    """Rank r fits its own batch of the workload's shape: the generator seed is r."""
    return W.workload(name, seed=rank)


def split_by_weight(b, world: int, P: int):
    """Contiguous shards of one batch's spectra, one per rank, balanced by the cumulative
    work weight P K_s (N_s + 2)^2 (spectra are independent: no exchange is needed, the
    results are gathered on the host). Returns [world + 1] spectrum boundaries."""
    w = P * b.K.astype(np.float64) * (b.n_poles.astype(np.float64) + 2.0) ** 2
    c = np.concatenate([[0.0], np.cumsum(w)])
    bounds = [0]
    for r in range(1, world):
        bounds.append(int(np.searchsorted(c, c[-1] * r / world, side="left")))
    bounds.append(b.S)
    return np.maximum.accumulate(np.array(bounds, dtype=np.int64))


def split_workload(name: str, rank: int, world: int):
    """Rank r's shard of the seed-0 batch (strong scaling: the total work is fixed)."""
    b = W.workload(name, seed=0)
    bounds = split_by_weight(b, world, SETTINGS[name][0])
    return b.subset(np.arange(bounds[rank], bounds[rank + 1]))


class RankReduce:
    """Barrier and max/sum over ranks (NCCL on the GPUs, gloo in the CPU tests); with
    one rank these are identities. No collective touches the fitted data."""

    def __init__(self, world: int, device=None):
        self.world = world
        self.device = device

    def _all_reduce(self, v: float, op) -> float:
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, v: float) -> float:
        if self.world == 1:
            return v
        import torch.distributed as dist
        return self._all_reduce(v, dist.ReduceOp.MAX)

    def sum(self, v: float) -> float:
        if self.world == 1:
            return v
        import torch.distributed as dist
        return self._all_reduce(v, dist.ReduceOp.SUM)

    def rate(self, work: float, seconds: float) -> float:
        """Whole-job throughput: all ranks' work over the slowest rank's time."""
        return self.sum(work) / self.max(seconds)


# ------------------------------------------------------------------ oracle timing (CPU)

def _oracle_chunk(job):
    """Oracle swarm generations of a chunk of spectra; returns (cand*K evaluated, compute seconds).
    The workload is built and the targets synthesised before the clock starts."""
    sys.path.insert(0, ROOT)
    import workloads as W_
    from oracle import dls, models, pso
    name, P, spectra, gens = job
    # the tabulated workload's generator draws every spectrum's noise at once (1 GB for all
    # 16384): its sample comes from a 64-spectrum batch of the same generator and shape
    full = W_.tabulated_batch(S=TAB_SAMPLE) if name == "tabulated_16384_k4096" else W_.workload(name)
    work, secs = 0, 0.0
    for s in spectra:
        b = full.subset([s])
        b.P = P
        re, im = models.synthesize(b)
        t0 = time.perf_counter()
        pso.pso(lambda th: dls.cost_population(b.omega, re, im, th)[0], int(b.n_poles[0]), float(b.lo[0]),
                float(b.hi[0]), b.P, gens - 1, seed=0, spectrum=int(s))
        secs += time.perf_counter() - t0
        work += b.P * gens * int(b.K[0])
    return work, secs


def oracle_rate(name: str, n_spectra: int, gens: int, procs: int, seed: int = 0):
    """cand*K/s of the oracle on a seeded sample of spectra of workload `name`, split over
    `procs` spawned processes: total work / the slowest process's compute time."""
    rng = np.random.default_rng(seed)
    S = {"single_hn_k50": 1, "mixed_1024": 1024, "hn_256_k2000": 256, "tabulated_16384_k4096": TAB_SAMPLE}[name]
    picks = [int(s) for s in rng.choice(S, min(n_spectra, S), replace=False)]
    chunks = [(name, SETTINGS[name][0], picks[i::procs], gens) for i in range(procs) if picks[i::procs]]
    # one BLAS thread per process, so `procs` is the number of cores used
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        res = pool.map(_oracle_chunk, chunks)
    work = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return work / wall, work, wall, len(chunks)


def cpu_model() -> str:
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        return next((l.split(":", 1)[1].strip() for l in txt.splitlines() if "Model name" in l), "")
    except Exception:
        return ""


def cpu_baseline(name: str, quick: bool):
    """The oracle on the host cores: one process, then one process per core."""
    cores = os.cpu_count() or 1
    n1, nall = (4, cores) if quick else (16, max(4 * cores, 32))
    if name == "tabulated_16384_k4096":      # ~9 s of oracle time per spectrum
        n1, nall = 1, min(2 * cores, TAB_SAMPLE)
    r1, _, t1, _ = oracle_rate(name, n1, 2, 1)
    ra, _, ta, used = oracle_rate(name, nall, 2, cores)
    src = (f"of a {TAB_SAMPLE}-spectrum batch drawn like {name}" if name == "tabulated_16384_k4096"
           else f"of {name}")
    return {"value": ra, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{nall} seeded spectra "
                      f"{src}, full population P={SETTINGS[name][0]}, 2 swarm "
                      f"generations (init + 1 update), numpy FP64 QR per candidate, {used} spawned processes; "
                      f"rate = total work / slowest process's compute time",
            "single_thread": {"value": r1, "sample": f"{n1} spectra, 1 process", "seconds": t1},
            "seconds": ta, "cpu_model": cpu_model()}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ GPU helpers

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(key: str):
    """DRAM bytes per pass recorded under `key` in the committed ncu summary, if the kernel
    source is unchanged since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        e = d.get(key)
        if e and e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


class Bench:
    """A workload on the device (targets synthesised by the library) and its fit calls."""

    def __init__(self, D, torch, dev, name: str, seed: int = 0, b=None):
        self.D, self.torch, self.dev, self.name = D, torch, dev, name
        self.P, self.iters, self.topk, self.polish_iters = SETTINGS[name]
        self.b = b if b is not None else W.workload(name, seed=seed)
        self.b.P = self.P
        self.seed = seed
        b = self.b
        tt = self.tt
        self.offsets_d, self.omega_d = tt(b.offsets, torch.int64), tt(b.omega)
        with D.Handle("fp64") as hs:
            noise = (tt(b.noise_re), tt(b.noise_im)) if b.noise_re is not None else (None, None)
            self.eps_re_d, self.eps_im_d = D.debye_synth_targets(
                hs, self.offsets_d, self.omega_d, tt(b.model, torch.int32), tt(b.params),
                tt(b.pole_offsets, torch.int64), tt(b.pole_tau), tt(b.pole_deps), *noise)
            D.debye_sync(hs)
        self.sp = D.Spectra(self.offsets_d, self.omega_d, self.eps_re_d, self.eps_im_d,
                            tt(b.n_poles, torch.int32), tt(b.lo), tt(b.hi),
                            np.ascontiguousarray(b.offsets, np.int64), np.ascontiguousarray(b.n_poles, np.int32))
        # F(N)-weighted and 54N-weighted cand*K of one full-population evaluation
        wK = b.K.astype(np.float64) * self.P
        self.candk_pass = float(wK.sum())
        self.alg_flops_pass = float(np.sum(wK * f_alg(b.n_poles)))

    def tt(self, a, dt=None):
        dt = dt or self.torch.float64
        return self.torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=self.dev)

    def fit(self, h, out=None, sp=None, iters=None, topk=None):
        return self.D.debye_fit_batch(h, sp or self.sp, P=self.P, iters=self.iters if iters is None else iters,
                                      seed=self.seed, polish_topk=self.topk if topk is None else topk,
                                      polish_iters=self.polish_iters, n_max=self.b.n_max, out=out)

    def population(self, seed):
        return self.torch.as_tensor(W.population(self.b, self.P, seed=seed), device=self.dev)


def timed_fits(bn: Bench, h, steps, warmup, flush, barrier=lambda: None, host_io=False, warm_iters=None):
    """Per-step CUDA-event times (ms) and cand*K per step of whole fits; L2 flushed between
    steps. warm_iters: generations of each warm-up fit (default: the workload's)."""
    torch, D = bn.torch, bn.D
    out = None
    for _ in range(warmup):
        out = bn.fit(h, out, iters=warm_iters)
    torch.cuda.synchronize()
    times, evals = [], []
    pinned = None
    if host_io:
        b = bn.b
        pinned = {k: torch.as_tensor(v).pin_memory() for k, v in (
            ("offsets", np.ascontiguousarray(b.offsets, np.int64)), ("omega", b.omega),
            ("eps_re", bn.eps_re_d.cpu().numpy()), ("eps_im", bn.eps_im_d.cpu().numpy()),
            ("n_poles", np.ascontiguousarray(b.n_poles, np.int32)), ("lo", b.lo), ("hi", b.hi))}
        dev_in = {k: torch.empty_like(v, device=bn.dev) for k, v in pinned.items()}
        res_host = {k: torch.empty(s, dtype=torch.float64).pin_memory()
                    for k, s in (("eps_inf", (b.S,)), ("d_eps", (b.S, b.n_max)), ("tau", (b.S, b.n_max)),
                                 ("final_cost", (b.S,)))}
    barrier()
    torch.cuda.synchronize()
    D.debye_launch_count(h, reset=True)
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        if host_io:
            for k in pinned:
                dev_in[k].copy_(pinned[k], non_blocking=True)
            spx = D.Spectra(dev_in["offsets"], dev_in["omega"], dev_in["eps_re"], dev_in["eps_im"],
                            dev_in["n_poles"], dev_in["lo"], dev_in["hi"], bn.sp.offsets_host, bn.sp.n_poles_host)
            out = bn.fit(h, out, spx)
            for k in res_host:
                res_host[k].copy_(out[k], non_blocking=True)
        else:
            out = bn.fit(h, out)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        evals.append(out["evals"].item())
    barrier()
    torch.cuda.synchronize()
    launches = D.debye_launch_count(h)
    h2d = sum(v.numel() * v.element_size() for v in pinned.values()) if host_io else 0
    d2h = sum(v.numel() * v.element_size() for v in res_host.values()) if host_io else 0
    return {"times": times, "evals": evals, "out": out, "h2d": h2d, "d2h": d2h, "launches": launches}


def profile(D, h, run):
    """Per-kind pass counts, milliseconds and issued FLOPs of `run()` with kernel timing on."""
    D.debye_profile_enable(h, True)
    run()
    import torch
    torch.cuda.synchronize()
    prof = D.debye_profile_read(h)
    D.debye_profile_enable(h, False)
    return prof


def roofline_mixed(bn: Bench, prof, traffic_key):
    """Roofline of the column-sum pass (the dominant kernel of every mixed evaluation) over the
    full-population passes of the profiled run: achieved = algorithmic FLOPs by the direct
    method's count F(N) = 4N + 2(N+2)^2 per cand*K (every unmasked candidate) / event time;
    frac_issued counts the pass's own float-float operations (54N per cand*K)."""
    n, ms, issued = prof["sums"]
    if n == 0 or ms <= 0:
        return None
    alg = n * bn.alg_flops_pass
    sec = ms * 1e-3
    ach = alg / sec / 1e12
    ach_issued = issued / sec / 1e12
    return {"bound": "alu", "kernel": "column-sum pass (k_pass<PH_SUMS, N>, one kernel per pole count)",
            "achieved": ach, "peak": PEAK_FP32, "unit": "TFLOP/s", "frac": ach / PEAK_FP32,
            "traffic": load_traffic(traffic_key), "passes": n, "ms_per_pass": ms / n,
            "cand_k_per_s": n * bn.candk_pass / sec,
            "flop_count": "F(N) = 4N + 2(N+2)^2 per cand*K (basis + unique Gram/RHS products of the "
                          "direct method), K-weighted over the batch",
            "achieved_issued": ach_issued, "frac_issued": ach_issued / PEAK_FP32,
            "issued_note": "the pass's own FP32 operations (54N per cand*K): float-float sums with "
                           "TwoSum/Dot2/Newton steps, i.e. the direct count plus precision overhead "
                           "minus the Gram products the partial-fraction identity removes",
            "peak_note": "FP32 ALU peak of measured-free unit counts: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz"}


def per_kind_ms(prof):
    return {k: v[1] for k, v in prof.items() if v[0]}


def fit_agreement(b, out_a, out_b):
    """Per-spectrum agreement of two fits of batch b (a: the arm under test, b: the FP64 fit):
    relative RMS between the fitted spectra, damped-cost ratio, fit error against the target."""
    from oracle import models as om
    re = b.extra.get("_re")
    rr, ratio, fe_a, fe_b = [], [], [], []
    for s in range(b.S):
        a, c = b.offsets[s], b.offsets[s + 1]
        N = int(b.n_poles[s])
        ea = om.multi_debye(b.omega[a:c], out_a["eps_inf"][s], out_a["d_eps"][s, :N], out_a["tau"][s, :N])
        eb = om.multi_debye(b.omega[a:c], out_b["eps_inf"][s], out_b["d_eps"][s, :N], out_b["tau"][s, :N])
        rr.append(float(np.linalg.norm(ea - eb) / np.linalg.norm(eb)))
        ratio.append(out_a["final_cost"][s] / out_b["final_cost"][s])
        if re is not None:
            tgt = re[0][a:c] - 1j * re[1][a:c]
            fe_a.append(float(np.linalg.norm(ea - tgt) / np.linalg.norm(tgt)))
            fe_b.append(float(np.linalg.norm(eb - tgt) / np.linalg.norm(tgt)))
    rr, ratio = np.array(rr), np.array(ratio)
    worse = ratio > 1 + 1e-6
    fail = (rr > 1e-4) & worse
    res = {"median_rel_rms": float(np.median(rr)), "frac_rel_rms_le_1e-4": float(np.mean(rr <= 1e-4)),
           "frac_cost_le_fp64": float(np.mean(~worse)), "n_fail_both": int(fail.sum()),
           "worst_cost_ratio": float(ratio.max()), "n_better_by_1e-6": int(np.sum(ratio < 1 - 1e-6))}
    if fe_a:
        fe_a, fe_b = np.array(fe_a), np.array(fe_b)
        res["fit_error_vs_target"] = {"median": float(np.median(fe_a)), "median_fp64": float(np.median(fe_b)),
                                      "mean": float(fe_a.mean()), "mean_fp64": float(fe_b.mean()),
                                      "frac_lower_than_fp64": float(np.mean(fe_a < fe_b))}
    return res


def host_out(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


# ------------------------------------------------------------------ extra configurations

def config_single_hn(D, torch, dev, flush, steps):
    """The paper-like single-target fit (HN, K = 50, N = 3, P = 64, 100 generations, FP64 plain
    method; mixed precision beside it): latency of one whole fit."""
    bn = Bench(D, torch, dev, "single_hn_k50")
    res = {"workload": "single_hn_k50: 1 HN spectrum (eps_inf 3.4, d_eps 2.7, tau0 8e-10 s, alpha 0.91, "
                       "beta 0.45), K=50 over 1e8-1e10 Hz, N=3, log10 tau in [-13,-6], P=64, 100 generations "
                       "after the first, top-8 x 50 L-BFGS polish, seed 0"}
    for prec in ("fp64", "mixed"):
        with D.Handle(prec) as h:
            r = timed_fits(bn, h, steps, 3, flush)
        res[prec] = {"ms_per_fit": float(np.mean(r["times"])), "value": sum(r["evals"]) / (sum(r["times"]) * 1e-3),
                     "unit": UNIT, "final_cost": float(r["out"]["final_cost"][0].item()), "steps": steps}
    return res


def config_hn256(D, torch, dev, flush, steps):
    """The differentiation workload: cost + VarPro gradient of 256 x 4096 fed-in candidates
    (K = 2000, N = 8) in both precisions, and the polish fit (top-32 x 50 L-BFGS, graph-captured)."""
    bn = Bench(D, torch, dev, "hn_256_k2000")
    b = bn.b
    th = bn.population(0)
    res = {"workload": "hn_256_k2000: 256 HN spectra, K=2000 over 1e6-1e10 Hz, N=8, 4096 fed-in candidates "
                       "per spectrum; cost+gradient of the population; fit = best 32 polished by 50 L-BFGS "
                       "iterations (CUDA graph)"}
    for prec in ("fp64", "mixed"):
        with D.Handle(prec) as h:
            cost, grad = D.debye_cost_grad(h, bn.sp, th)
            torch.cuda.synchronize()
            t = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                D.debye_cost_grad(h, bn.sp, th, cost=cost, grad=grad)
                e1.record()
                torch.cuda.synchronize()
                t.append(e0.elapsed_time(e1))
            prof = profile(D, h, lambda: D.debye_cost_grad(h, bn.sp, th, cost=cost, grad=grad))
            entry = {"cost_grad_ms": float(np.mean(t)),
                     "cost_grad_value": bn.candk_pass / (np.mean(t) * 1e-3), "unit": UNIT,
                     "per_kind_ms": per_kind_ms(prof)}
            if prec == "mixed":
                n, ms, issued = prof["sums"]
                if n:
                    entry["sums_grad_pass"] = {"ms": ms / n, "achieved_issued": issued / (ms * 1e-3) / 1e12,
                                               "frac_issued": issued / (ms * 1e-3) / 1e12 / PEAK_FP32,
                                               "note": "pass with the derivative sums, its own 103N FP32 "
                                                       "operations per cand*K"}
                r = timed_fits(bn, h, steps, 1, flush)
                entry["fit_ms"] = float(np.mean(r["times"]))
                entry["fit_value"] = sum(r["evals"]) / (sum(r["times"]) * 1e-3)
            res[prec] = entry
    return res


def config_tabulated(D, torch, dev, flush):
    """The tabulated workload at full size: 16384 spectra x 4096 samples, N = 20, P = 512,
    100 generations, top-8 x 50 polish; one warm-up fit of one generation (allocation,
    graph capture paths), one timed fit; the column-sum pass's roofline from a profiled
    three-generation fit without the polish (its full-population passes are identical in every
    generation)."""
    bn = Bench(D, torch, dev, "tabulated_16384_k4096")
    res = {"workload": "tabulated_16384_k4096: 16384 spectra (40 random Debye poles + Jonscher tail, 1% "
                       "Gaussian noise), K=4096 over 1e5-1e10 Hz, N=20, P=512, 100 generations after the "
                       "first, top-8 x 50 L-BFGS polish, mixed precision"}
    with D.Handle("mixed") as h:
        r = timed_fits(bn, h, 1, 1, flush, warm_iters=1)
        res["ms_per_step"] = float(r["times"][0])
        res["value"] = r["evals"][0] / (r["times"][0] * 1e-3)
        res["unit"] = UNIT
        res["cand_k_per_step"] = r["evals"][0]
        out_direct = host_out(r["out"])     # before the profiled run reuses the output buffers
        prof = profile(D, h, lambda: bn.fit(h, r["out"], iters=2, topk=0))
        res["roofline"] = roofline_mixed(bn, prof, "sums_tabulated_16384_k4096")
        res["per_kind_ms_3_generations"] = per_kind_ms(prof)
    del r
    with D.Handle("mixed_table") as h:
        rt = timed_fits(bn, h, 1, 1, flush, warm_iters=1)
        res["mixed_table"] = {"ms_per_step": float(rt["times"][0]), "unit": UNIT,
                              "value": rt["evals"][0] / (rt["times"][0] * 1e-3),
                              "speedup_over_direct_mixed": res["ms_per_step"] / float(rt["times"][0]),
                              "fit_agreement_vs_direct_mixed": {
                                  k: v for k, v in fit_agreement(bn.b, host_out(rt["out"]), out_direct).items()
                                  if k != "fit_error_vs_target"}}
        prof = profile(D, h, lambda: bn.fit(h, rt["out"], iters=2, topk=0))
        res["mixed_table"]["per_kind_ms_3_generations"] = per_kind_ms(prof)
    return res


def fp64_arm(D, torch, bn: Bench, precision: str, steps: int, flush, red, mixed_value):
    """An FP64 evaluator on the headline fit: rate over `steps` timed fits (one warm-up), the
    roofline of its Gram pass (one full-population evaluation, kernel timing on)."""
    h = D.Handle(precision)
    D.debye_autotune(h, bn.sp, bn.population(2))
    r = timed_fits(bn, h, steps, 1, flush, red.barrier)
    v = red.sum(sum(r["evals"])) / red.max(sum(r["times"]) * 1e-3)
    out = host_out(r["out"])
    th_pop = bn.population(1)
    D.debye_eval_population(h, bn.sp, th_pop)
    pd = profile(D, h, lambda: D.debye_eval_population(h, bn.sp, th_pop))
    h.close()
    n_g, ms_g, fl_g = pd["gram"]
    what = ("FP64 Gram pass (k_pass<PH_GRAM, N>), 4N + 2(N+2)^2 FP64 FLOPs per cand*K" if precision == "fp64" else
            "FP64 column-sum pass (k_pass<PH_GRAM_SUMS, N>), 8N + 2 FP64 FLOPs per cand*K")
    ach = fl_g / (ms_g * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": what, "unit": "TFLOP/s", "achieved": ach, "peak": PEAK_FP64,
            "frac": ach / PEAK_FP64, "ms_per_pass": ms_g / max(n_g, 1),
            "cand_k_per_s_per_pass": bn.candk_pass / (ms_g * 1e-3 / max(n_g, 1)),
            "peak_note": "nominal GB300 FP64 rate 1.25 TFLOP/s (an FMA-chain probe measured 1.195)",
            "per_kind_ms_one_evaluation": per_kind_ms(pd)}
    return ({"value": v, "unit": UNIT, "ms_per_step": float(np.mean(r["times"])), "steps": steps,
             "speedup_mixed_over_this": mixed_value / v, "roofline": roof}, out)


def table_arm(D, torch, bn: Bench, steps: int, warmup: int, flush, red, mixed_value, out_mixed, out_fp64):
    """The mixed path with the column sums read from per-spectrum Chebyshev tables
    (DEBYE_PREC_MIXED_TABLE) on the headline fit: rate over `steps` timed fits, the
    per-kind breakdown of one fit (kernel timing on), and the agreement of its fitted
    spectra with the FP64 fit and with the direct mixed fit."""
    h = D.Handle("mixed_table")
    tuned = D.debye_autotune(h, bn.sp, bn.population(2))
    r = timed_fits(bn, h, steps, warmup, flush, red.barrier)
    v = red.sum(sum(r["evals"])) / red.max(sum(r["times"]) * 1e-3)
    out = host_out(r["out"])
    prof = profile(D, h, lambda: bn.fit(h, r["out"]))
    h.close()
    res = {"value": v, "unit": UNIT, "ms_per_step": float(np.mean(r["times"])), "steps": steps,
           "speedup_over_direct_mixed": v / mixed_value, "autotune": tuned, "per_kind_ms": per_kind_ms(prof),
           "what": "column sums S, a^T b and their theta derivatives of every pole interpolated from "
                   "per-spectrum Chebyshev tables (0.2-decade segments, 12 coefficients, built once per "
                   "fit from float-float node sums); same solve, cost and search as the direct mixed path"}
    if out_fp64 is not None:
        res["fit_agreement"] = fit_agreement(bn.b, out, out_fp64)
    res["fit_agreement_vs_direct_mixed"] = {
        k: v_ for k, v_ in fit_agreement(bn.b, out, out_mixed).items() if k != "fit_error_vs_target"}
    return res


# ------------------------------------------------------------------ main

def main():
    global WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-table", action="store_true", help="skip the Chebyshev-table arm")
    ap.add_argument("--split", action="store_true",
                    help="with N > 1: split the one seed-0 batch across the ranks by work weight (strong "
                         "scaling) instead of one replica batch per rank (weak scaling, the default)")
    ap.add_argument("--configs", default="all", help="extra workloads: all, none or a comma list of "
                    + ", ".join(EXTRA_CONFIGS))
    ap.add_argument("--iters", type=int, default=None, help="swarm generations (default: the workload's)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(SETTINGS))
    ap.add_argument("--kernel-case", type=int, default=0, metavar="S",
                    help="profiling case: evaluate the first S spectra of the workload at full "
                         "population twice (debye_eval_population) and exit")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp64_sums", "mixed_table"],
                    help="precision of --kernel-case and --fit-case")
    ap.add_argument("--fit-case", action="store_true",
                    help="profiling case: one short warm-up fit and one whole fit of the workload in --precision, "
                         "then exit")
    ap.add_argument("--kernel-n", type=int, default=0, metavar="N",
                    help="--kernel-case: fit every spectrum with N poles (one pass kernel fills the GPU)")
    args = ap.parse_args()

    WORKLOAD = args.workload
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    configs = [] if args.configs == "none" else (list(EXTRA_CONFIGS) if args.configs == "all"
                                                else [c for c in args.configs.split(",") if c])

    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.kernel_case:
        return kernel_case(args.kernel_case, args.precision, SETTINGS[WORKLOAD][0], args.kernel_n)
    if args.fit_case:
        return fit_case(args.precision)

    # the oracle baselines run first, in spawned processes, before any CUDA call
    cpu, cpu_tab = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(WORKLOAD, quick=False)
        if "tabulated_16384_k4096" in configs:
            cpu_tab = cpu_baseline("tabulated_16384_k4096", quick=False)

    import torch
    import torch.distributed as dist
    from paper_2109_01928_gb300 import debyefit as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://", device_id=dev)
    red = RankReduce(world, dev)

    bsel = split_workload(WORKLOAD, rank, world) if args.split else replica_workload(WORKLOAD, rank)
    bn = Bench(D, torch, dev, WORKLOAD, seed=0 if args.split else rank, b=bsel)
    if args.iters is not None:
        bn.iters = args.iters
    b = bn.b
    desc = workload_desc(b, bn.iters)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    hm = D.Handle("mixed")
    # pick the work layout on this batch before timing (project autotuner)
    tuned = D.debye_autotune(hm, bn.sp, bn.population(2))
    with ClockSampler(local) as clk:
        rm = timed_fits(bn, hm, args.steps, args.warmup, flush, red.barrier)
    clocks = clk.summary()
    value = red.sum(sum(rm["evals"])) / red.max(sum(rm["times"]) * 1e-3)
    out_mixed = host_out(rm["out"])

    # end to end through the C ABI with host buffers (pinned H2D in, D2H of the result)
    re2e = timed_fits(bn, hm, max(1, args.steps // 2), 1, flush, red.barrier, host_io=True)
    e2e_value = red.sum(sum(re2e["evals"])) / red.max(sum(re2e["times"]) * 1e-3)

    # live kernel timing of one step (events on the launching stream; graph capture off)
    prof = profile(D, hm, lambda: bn.fit(hm, rm["out"]))
    roof = roofline_mixed(bn, prof, "sums_mixed_1024")
    roof["per_kind_ms"] = per_kind_ms(prof)
    roof["step_frac"] = value / world * bn.alg_flops_pass / bn.candk_pass / 1e12 / PEAK_FP32

    # one batched evaluation of the whole population vs one launch sequence per spectrum
    batching = None
    if not args.no_fp64 and world == 1:
        th_pop = bn.population(1)
        per_spec = []
        for s in range(b.S):
            a_, c_ = int(b.offsets[s]), int(b.offsets[s + 1])
            per_spec.append((D.Spectra(bn.tt(np.array([0, c_ - a_]), torch.int64), bn.omega_d[a_:c_],
                                       bn.eps_re_d[a_:c_], bn.eps_im_d[a_:c_], bn.tt(b.n_poles[s:s + 1], torch.int32),
                                       bn.tt(b.lo[s:s + 1]), bn.tt(b.hi[s:s + 1]), np.array([0, c_ - a_], np.int64),
                                       np.ascontiguousarray(b.n_poles[s:s + 1], np.int32)),
                             th_pop[s:s + 1].contiguous()))
        batching = {}
        for prec in ("mixed", "fp64"):
            with D.Handle(prec) as hb:
                D.debye_eval_population(hb, bn.sp, th_pop)        # warm-up (workspaces)
                for spx, thx in per_spec[:4]:
                    D.debye_eval_population(hb, spx, thx)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                D.debye_eval_population(hb, bn.sp, th_pop)
                e1.record()
                torch.cuda.synchronize()
                t_batched = e0.elapsed_time(e1)
                e0.record()
                for spx, thx in per_spec:
                    D.debye_eval_population(hb, spx, thx)
                e1.record()
                torch.cuda.synchronize()
                t_each = e0.elapsed_time(e1)
            batching[prec] = {"batched_ms": t_batched, "per_spectrum_ms": t_each,
                              "batched_candK_per_s": bn.candk_pass / (t_batched * 1e-3),
                              "per_spectrum_candK_per_s": bn.candk_pass / (t_each * 1e-3)}

    # the FP64 GPU evaluators on the same fit: the plain method (direct Gram pass) and the Gram
    # from FP64 column sums; their rooflines, and the agreement of the fitted spectra
    fp64, fp64_sums = None, None
    if not args.no_fp64:
        b.extra["_re"] = (bn.eps_re_d.cpu().numpy(), bn.eps_im_d.cpu().numpy())
        fp64, out_fp64 = fp64_arm(D, torch, bn, "fp64", args.fp64_steps, flush, red, value)
        fp64["fit_agreement"] = fit_agreement(b, out_mixed, out_fp64)
        # noise floor of the criterion: the FP64 fit against itself with the damping moved by 1e-9
        lam = D.default_options().lam_search * (1 + CTL_REL)
        with D.Handle("fp64", lam_search=lam, lam_final=lam) as hc:
            out_ctl = host_out(bn.fit(hc))
        ctl = fit_agreement(b, out_ctl, out_fp64)
        fp64["fit_agreement"]["fp64_control"] = {
            "what": f"the FP64 fit with lam_search = lam_final = 1e-3 (1 + {CTL_REL:g}) against the FP64 fit: "
                    "the same criteria, showing how many spectra a 1e-9 change of the problem moves past them",
            **{k: ctl[k] for k in ("n_fail_both", "worst_cost_ratio", "frac_rel_rms_le_1e-4", "median_rel_rms")}}
        fp64_sums, out_sums = fp64_arm(D, torch, bn, "fp64_sums", args.fp64_steps, flush, red, value)
        fp64_sums["fit_agreement_vs_fp64"] = {
            k: v for k, v in fit_agreement(b, out_sums, out_fp64).items() if k != "fit_error_vs_target"}
    hm.close()
    table = None
    if not args.no_table:
        table = table_arm(D, torch, bn, args.steps, args.warmup, flush, red, value, out_mixed,
                          None if args.no_fp64 else out_fp64)

    extra = {}
    if rank == 0 and world == 1:
        if "single_hn_k50" in configs:
            extra["single_hn_k50"] = config_single_hn(D, torch, dev, flush, 10)
        if "hn_256_k2000" in configs:
            extra["hn_256_k2000"] = config_hn256(D, torch, dev, flush, 3)
        if "tabulated_16384_k4096" in configs:
            del bn, flush
            torch.cuda.empty_cache()
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
            extra["tabulated_16384_k4096"] = config_tabulated(D, torch, dev, flush)
            if cpu_tab:
                extra["tabulated_16384_k4096"]["cpu_baseline"] = cpu_tab

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(rm["times"])), "higher_is_better": True,
        "scaling": "strong" if args.split else "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded HN/CC/CD/Jonscher/CRIM spectra, targets synthesised on the device)",
        "config": {"workload": desc,
                   "precision": "mixed (float-float column sums, exact Gram identity, FP32 factor refined "
                                "in float-float)",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": (f"weight-balanced split of one batch x{world}" if args.split
                                   else f"replicas x{world}")},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": re2e["h2d"],
                "d2h_bytes_per_step": re2e["d2h"]},
        "gpu_launches": rm["launches"],
        "autotune": tuned,
        "roofline": roof,
        "cpu_baseline": cpu,
        "fp64_plain": fp64,
        "fp64_sums": fp64_sums,
        "mixed_table": table,
        "eval_batching": batching,
        "configs": extra,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def kernel_case(S: int, precision: str, P: int, n_poles: int = 0):
    """A small fixed case for kernel profilers: one workload subset, two evaluations."""
    import torch
    from paper_2109_01928_gb300 import debyefit as D
    b = W.workload(WORKLOAD).subset(np.arange(S))
    if n_poles:
        b.n_poles = np.full(b.S, n_poles, dtype=np.int32)
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    om, offs = tt(b.omega), tt(b.offsets, torch.int64)
    with D.Handle(precision) as h:
        noise = (tt(b.noise_re), tt(b.noise_im)) if b.noise_re is not None else (None, None)
        er, ei = D.debye_synth_targets(h, offs, om, tt(b.model, torch.int32), tt(b.params),
                                       tt(b.pole_offsets, torch.int64), tt(b.pole_tau), tt(b.pole_deps), *noise)
        sp = D.Spectra(offs, om, er, ei, tt(b.n_poles, torch.int32), tt(b.lo), tt(b.hi),
                       np.ascontiguousarray(b.offsets), np.ascontiguousarray(b.n_poles, np.int32))
        b.P = P
        th = torch.as_tensor(W.population(b, P, seed=0), device="cuda")
        for _ in range(2):
            c = D.debye_eval_population(h, sp, th)
        D.debye_sync(h)
    print(json.dumps({"kernel_case": WORKLOAD, "spectra": S, "P": P, "n_poles": n_poles, "precision": precision,
                      "mean_cost": float(c.mean())}))


def fit_case(precision: str):
    """A fixed case for launch-list captures: the workload's targets, one short warm-up fit
    (2 generations, 2 polish iterations) and one whole fit on one handle."""
    import torch
    from paper_2109_01928_gb300 import debyefit as D
    bn = Bench(D, torch, torch.device("cuda", 0), WORKLOAD)
    with D.Handle(precision) as h:
        out = D.debye_fit_batch(h, bn.sp, P=bn.P, iters=2, seed=0, polish_topk=bn.topk, polish_iters=2,
                                n_max=bn.b.n_max)
        out = bn.fit(h, out)
        D.debye_sync(h)
    print(json.dumps({"fit_case": WORKLOAD, "precision": precision, "sum_final_cost": float(out["final_cost"].sum())}))


def workload_desc(b, iters) -> str:
    """The timed workload, as both arms name it in `config`."""
    P, _, topk, pit = SETTINGS[WORKLOAD]
    return (f"{WORKLOAD}: {b.S} spectra, K {int(b.K.min())}-{int(b.K.max())} (sum {int(b.K.sum())}), "
            f"N {int(b.n_poles.min())}-{int(b.n_poles.max())}, P={P}, {iters} swarm generations after the "
            f"first, top-{topk} x {pit} L-BFGS polish")


def reference_arm(args, rank, world):
    """The FP64 oracle on the host cores, on bounded samples of the same workload."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    times, work = [], []
    used = cores
    for i in range(args.warmup + args.steps):
        r, w, t, used = oracle_rate(WORKLOAD, max(cores, 4), 2, cores, seed=i)
        if i >= args.warmup:
            times.append(t)
            work.append(w)
    value = sum(work) / sum(times)
    cpu = {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"per step {max(cores, 4)} seeded spectra of {WORKLOAD}, P={SETTINGS[WORKLOAD][0]}, "
                     f"2 swarm generations"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": workload_desc(W.workload(WORKLOAD), SETTINGS[WORKLOAD][1]),
                                 "precision": "FP64 oracle (numpy, host cores)",
                                 "sample": cpu["sample"], "parallelism": f"{used} host processes"},
                      "cpu_baseline": cpu,
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    main()
