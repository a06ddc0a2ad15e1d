"""Throughput of batched multi-Debye fitting on GB300.

One step = one debye_fit_batch over the whole workload: seeded particle swarm
(every generation evaluates the damped least-squares cost of every particle),
L-BFGS polish of the best personal bests, final FP64 re-solve. The metric is
candidate evaluations x frequency samples per second (cand*K/s), counted on the
device over swarm and polish evaluations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank fits its own batch of the same shape (seed =
rank): the spectra are independent, so there is no data-path collective, and
the value is the total over ranks divided by the slowest rank's time (weak
scaling). Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
TOPK, POLISH_ITERS = 8, 50
METRIC = "candidate cost evals x K per sec (batched mixed-precision fit)"
UNIT = "cand*K/s"
FP32_LANES_PER_SM, SMS, SM_MAX_MHZ = 128, 152, 2070.0
KERNEL_SOURCES = ["paper_2109_01928_gb300/csrc/eval.cuh", "paper_2109_01928_gb300/csrc/common.cuh"]


# ------------------------------------------------------------------ replicas (one process per GPU)

def replica_workload(name: str, rank: int):
    """Rank r fits its own batch of the workload's shape: the generator seed is r."""
    return W.workload(name, seed=rank)


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
    full = W_.workload(name)
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


def oracle_rate(n_spectra: int, gens: int, procs: int, seed: int = 0):
    """cand*K/s of the oracle on a seeded sample of spectra, split over `procs` spawned
    processes: total work / the slowest process's compute time."""
    rng = np.random.default_rng(seed)
    S = W.workload(WORKLOAD).S
    picks = [int(s) for s in rng.choice(S, n_spectra, replace=False)]
    chunks = [(WORKLOAD, SETTINGS[WORKLOAD][0], picks[i::procs], gens) for i in range(procs) if picks[i::procs]]
    # one BLAS thread per process, so `procs` is the number of cores used
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        res = pool.map(_oracle_chunk, chunks)
    work = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return work / wall, work, wall


def cpu_baseline(quick: bool):
    cores = os.cpu_count() or 1
    b = W.workload(WORKLOAD)
    heavy = float(np.mean(b.K)) * SETTINGS[WORKLOAD][0] > 3e5   # per-spectrum oracle work
    n1, nall = (4, cores) if (quick or heavy) else (16, max(4 * cores, 32))
    r1, w1, t1 = oracle_rate(n1, 2, 1)
    ra, wa, ta = oracle_rate(nall, 2, cores)
    try:
        model = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        model = next((l.split(":", 1)[1].strip() for l in model.splitlines() if "Model name" in l), "")
    except Exception:
        model = ""
    return {"value": ra, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nall} seeded spectra of {WORKLOAD}, full population P={SETTINGS[WORKLOAD][0]}, 2 swarm generations "
                      f"(init + 1 update), numpy FP64 QR per candidate, {cores} spawned processes; "
                      f"rate = total work / slowest process's compute time",
            "single_thread": {"value": r1, "sample": f"{n1} spectra, 1 process", "seconds": t1},
            "seconds": ta, "cpu_model": model}


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


# ------------------------------------------------------------------ GPU arm

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kind: str):
    """DRAM bytes per launch of kernel `kind` from the committed ncu summary, if the kernel
    source is unchanged since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        e = d.get(kind)
        if e and e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def main():
    global WORKLOAD, TOPK, POLISH_ITERS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--iters", type=int, default=None, help="swarm generations (default: the workload's)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(SETTINGS))
    ap.add_argument("--kernel-case", type=int, default=0, metavar="S",
                    help="profiling case: evaluate the first S spectra of the workload at full "
                         "population twice (debye_eval_population) and exit")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of --kernel-case")
    ap.add_argument("--kernel-n", type=int, default=0, metavar="N",
                    help="--kernel-case: fit every spectrum with N poles (one pass kernel fills the GPU)")
    args = ap.parse_args()

    WORKLOAD = args.workload
    P_w, iters_w, TOPK, POLISH_ITERS = SETTINGS[WORKLOAD]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.kernel_case:
        return kernel_case(args.kernel_case, args.precision, P_w, args.kernel_n)

    # the oracle baseline runs first, in spawned processes, before any CUDA call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(quick=False)

    import torch
    import torch.distributed as dist
    from oracle import dls  # noqa: F401  (only for the fit-agreement statistics below)
    from paper_2109_01928_gb300 import debyefit as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://", device_id=dev)

    red = RankReduce(world, dev)
    barrier, max_over_ranks, sum_over_ranks = red.barrier, red.max, red.sum

    b = replica_workload(WORKLOAD, rank)
    b.P = P_w
    iters = iters_w if args.iters is None else args.iters
    S = b.S
    nmax = b.n_max
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    offsets_d = tt(b.offsets, torch.int64)
    omega_d = tt(b.omega)
    # target synthesis (Eqs. 4-6) on the device, once, outside the timed region
    with D.Handle("fp64") as hs:
        noise = (tt(b.noise_re), tt(b.noise_im)) if b.noise_re is not None else (None, None)
        eps_re_d, eps_im_d = D.debye_synth_targets(hs, offsets_d, omega_d, tt(b.model, torch.int32),
                                                    tt(b.params), tt(b.pole_offsets, torch.int64),
                                                    tt(b.pole_tau), tt(b.pole_deps), *noise)
        D.debye_sync(hs)
    sp = D.Spectra(offsets_d, omega_d, eps_re_d, eps_im_d, tt(b.n_poles, torch.int32), tt(b.lo), tt(b.hi),
                   np.ascontiguousarray(b.offsets, np.int64), np.ascontiguousarray(b.n_poles, np.int32))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def fit_once(h, out=None, spx=None):
        return D.debye_fit_batch(h, spx or sp, P=b.P, iters=iters, seed=rank, polish_topk=TOPK,
                                 polish_iters=POLISH_ITERS, n_max=nmax, out=out)

    def timed_steps(h, steps, warmup, host_io=False):
        """Per-step CUDA-event times (ms) and cand*K per step; L2 flushed between steps."""
        out = None
        for _ in range(warmup):
            out = fit_once(h, out)
        torch.cuda.synchronize()
        times, evals = [], []
        pinned = None
        if host_io:
            pinned = {k: torch.as_tensor(v).pin_memory() for k, v in (
                ("offsets", np.ascontiguousarray(b.offsets, np.int64)), ("omega", b.omega),
                ("eps_re", eps_re_d.cpu().numpy()), ("eps_im", eps_im_d.cpu().numpy()),
                ("n_poles", np.ascontiguousarray(b.n_poles, np.int32)), ("lo", b.lo), ("hi", b.hi))}
            dev_in = {k: torch.empty_like(v, device=dev) for k, v in pinned.items()}
            res_host = {k: torch.empty(s, dtype=torch.float64).pin_memory()
                        for k, s in (("eps_inf", (S,)), ("d_eps", (S, nmax)), ("tau", (S, nmax)),
                                     ("final_cost", (S,)))}
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
                                dev_in["n_poles"], dev_in["lo"], dev_in["hi"], sp.offsets_host,
                                sp.n_poles_host)
                out = fit_once(h, out, spx)
                for k in res_host:
                    res_host[k].copy_(out[k], non_blocking=True)
            else:
                out = fit_once(h, out)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            evals.append(out["evals"].item())
        barrier()
        torch.cuda.synchronize()
        timed_steps.launches = D.debye_launch_count(h)
        h2d = sum(v.numel() * v.element_size() for v in pinned.values()) if host_io else 0
        d2h = sum(v.numel() * v.element_size() for v in res_host.values()) if host_io else 0
        return times, evals, out, h2d, d2h

    hm = D.Handle("mixed")
    # pick the work layout on this batch before timing (project autotuner)
    th_tune = torch.as_tensor(W.population(b, b.P, seed=2), device=dev)
    tuned = D.debye_autotune(hm, sp, th_tune)
    del th_tune
    with ClockSampler(local) as clk:
        times, evals, out_mixed, _, _ = timed_steps(hm, args.steps, args.warmup)
    clocks = clk.summary()
    t_total = max_over_ranks(sum(times) * 1e-3)
    work = sum_over_ranks(sum(evals))
    value = work / t_total
    launches = timed_steps.launches

    # end to end through the C ABI with host buffers (pinned H2D in, D2H of the result)
    e_times, e_evals, _, h2d, d2h = timed_steps(hm, max(1, args.steps // 2), 1, host_io=True)
    e2e_value = sum_over_ranks(sum(e_evals)) / max_over_ranks(sum(e_times) * 1e-3)

    # live kernel timing of one step (events on the launching stream; graph capture off)
    D.debye_profile_enable(hm, True)
    fit_once(hm, out_mixed)
    torch.cuda.synchronize()
    prof = D.debye_profile_read(hm)
    D.debye_profile_enable(hm, False)
    kind = max(("gram", "refine", "sums"), key=lambda k: prof[k][1])
    n_l, ms_l, fl = prof[kind]
    achieved = fl / (ms_l * 1e-3) / 1e12 if ms_l > 0 else 0.0
    peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = load_traffic(kind)
    # F(N) = 4N + 2(N+2)^2 per cand*K (basis + unique Gram products), averaged over the batch
    fN = float(np.sum(b.K * b.P * (4 * b.n_poles + 2 * (b.n_poles + 2.0) ** 2)) / np.sum(b.K * b.P))
    step_fp32 = value / world * fN / 1e12

    # one batched evaluation of the whole population vs one launch sequence per spectrum
    batching = None
    if not args.no_fp64 and world == 1:
        th_pop = torch.as_tensor(W.population(b, b.P, seed=1), device=dev)
        per_spec = []
        for s in range(S):
            a_, c_ = int(b.offsets[s]), int(b.offsets[s + 1])
            per_spec.append((D.Spectra(tt(np.array([0, c_ - a_]), torch.int64), omega_d[a_:c_], eps_re_d[a_:c_],
                                       eps_im_d[a_:c_], tt(b.n_poles[s:s + 1], torch.int32), tt(b.lo[s:s + 1]),
                                       tt(b.hi[s:s + 1]), np.array([0, c_ - a_], np.int64),
                                       np.ascontiguousarray(b.n_poles[s:s + 1], np.int32)),
                             th_pop[s:s + 1].contiguous()))
        batching = {}
        for prec in ("mixed", "fp64"):
            with D.Handle(prec) as hb:
                D.debye_eval_population(hb, sp, th_pop)        # warm-up (workspaces)
                for spx, thx in per_spec[:4]:
                    D.debye_eval_population(hb, spx, thx)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                D.debye_eval_population(hb, sp, th_pop)
                e1.record()
                torch.cuda.synchronize()
                t_batched = e0.elapsed_time(e1)
                t0 = time.perf_counter()
                e0.record()
                for spx, thx in per_spec:
                    D.debye_eval_population(hb, spx, thx)
                e1.record()
                torch.cuda.synchronize()
                t_each = e0.elapsed_time(e1)
            candk = float(b.P * b.K.sum())
            batching[prec] = {"batched_ms": t_batched, "per_spectrum_ms": t_each,
                              "batched_candK_per_s": candk / (t_batched * 1e-3),
                              "per_spectrum_candK_per_s": candk / (t_each * 1e-3)}

    # the plain FP64 GPU evaluator on the same workload, and agreement of the fitted spectra
    fp64 = None
    if not args.no_fp64:
        hd = D.Handle("fp64")
        th_tune = torch.as_tensor(W.population(b, b.P, seed=2), device=dev)
        D.debye_autotune(hd, sp, th_tune)
        del th_tune
        d_times, d_evals, out_fp64, _, _ = timed_steps(hd, 1, 1)
        d_value = sum_over_ranks(sum(d_evals)) / max_over_ranks(sum(d_times) * 1e-3)
        from oracle import models as om
        rr, better = [], 0
        for s in range(S):
            a, c = b.offsets[s], b.offsets[s + 1]
            N = int(b.n_poles[s])
            em = om.multi_debye(b.omega[a:c], out_mixed["eps_inf"][s].item(),
                                out_mixed["d_eps"][s, :N].cpu().numpy(), out_mixed["tau"][s, :N].cpu().numpy())
            ed = om.multi_debye(b.omega[a:c], out_fp64["eps_inf"][s].item(),
                                out_fp64["d_eps"][s, :N].cpu().numpy(), out_fp64["tau"][s, :N].cpu().numpy())
            rr.append(float(np.linalg.norm(em - ed) / np.linalg.norm(ed)))
            better += out_mixed["final_cost"][s].item() <= out_fp64["final_cost"][s].item() * (1 + 1e-6)
        rr = np.array(rr)
        fp64 = {"value": d_value, "unit": UNIT, "ms_per_step": sum(d_times) / len(d_times),
                "speedup_mixed_over_fp64": value / d_value,
                "fit_agreement": {"median_rel_rms": float(np.median(rr)),
                                  "frac_rel_rms_le_1e-4": float(np.mean(rr <= 1e-4)),
                                  "frac_mixed_cost_le_fp64": better / S}}
        hd.close()

    hm.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded HN/CC/CD/Jonscher/CRIM spectra, targets synthesised on the device)",
        "config": {"workload": workload_desc(b, iters),
                   "precision": "mixed (float-float column sums, exact Gram identity, FP32 factor refined "
                                "in float-float)",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "autotune": {"cands_per_block": tuned},
        "roofline": {"bound": "alu", "kernel": kind, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "passes": n_l, "ms_per_pass": ms_l / max(n_l, 1),
                     "pass_note": "one pass = the concurrent launches of the pass kernel for every "
                                  "pole count (one kernel per N on forked streams), timed fork to join; "
                                  "full-population passes only (the line search's masked passes are "
                                  "timed under *_masked)",
                     "peak_note": "FP32 FMA pipe: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz",
                     "step_fp32_tflops": step_fp32, "step_fp32_frac": step_fp32 / peak,
                     "per_kind_ms": {k: v[1] for k, v in prof.items()}},
        "cpu_baseline": cpu,
        "fp64_plain": fp64,
        "eval_batching": batching,
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


def workload_desc(b, iters) -> str:
    """The timed workload, as both arms name it in `config`."""
    return (f"{WORKLOAD}: {b.S} spectra, K {int(b.K.min())}-{int(b.K.max())} (sum {int(b.K.sum())}), "
            f"N {int(b.n_poles.min())}-{int(b.n_poles.max())}, P={b.P}, {iters} swarm generations after the "
            f"first, top-{TOPK} x {POLISH_ITERS} L-BFGS polish")


def reference_arm(args, rank, world):
    """The FP64 oracle on the host cores, on bounded samples of the same workload."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    times, work = [], []
    for i in range(args.warmup + args.steps):
        r, w, t = oracle_rate(max(cores, 4), 2, cores, seed=i)
        if i >= args.warmup:
            times.append(t)
            work.append(w)
    value = sum(work) / sum(times)
    cpu = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"per step {max(cores, 4)} seeded spectra of {WORKLOAD}, P={SETTINGS[WORKLOAD][0]}, "
                     f"2 swarm generations"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": workload_desc(W.workload(WORKLOAD), SETTINGS[WORKLOAD][1]),
                                 "precision": "FP64 oracle (numpy, host cores)",
                                 "sample": cpu["sample"], "parallelism": f"{cores} host processes"},
                      "cpu_baseline": cpu,
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    main()
