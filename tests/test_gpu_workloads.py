"""Full-size workloads on the GPU, checked on sampled outputs the oracle computes
one by one: the 256-spectrum K=2000 differentiation workload (costs, gradients,
polish-only fit) and the 16384-spectrum K=4096 tabulated workload (costs), in FP64
and in mixed precision with direct and tabulated column sums."""
import numpy as np
import pytest

import fitcheck
import workloads as W
from oracle import dls, fit, models, varpro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COST_TOL = {"fp64": 1e-10, "mixed": 1e-5, "mixed_table": 1e-5}
GRAD_TOL = {"fp64": 1e-8, "mixed": 1e-4, "mixed_table": 1e-4}


@pytest.fixture(scope="module")
def D():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2109_01928_gb300 import debyefit
    debyefit.lib()
    return debyefit


@pytest.fixture(scope="module")
def hn256():
    b = W.workload("hn_256_k2000")
    re, im = models.synthesize(b)
    return b, re, im


def _spectra(D, b, re, im):
    return D.make_spectra(b.offsets, b.omega, re, im, b.n_poles, b.lo, b.hi, device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_table"])
def test_hn256_cost_grad_sampled(D, hn256, prec):
    b, re, im = hn256
    th = W.population(b, 4096, seed=0)
    with D.Handle(prec) as h:
        cost, grad = D.debye_cost_grad(h, _spectra(D, b, re, im), torch.as_tensor(th, device="cuda"))
        D.debye_sync(h)
    cost, grad = cost.cpu().numpy(), grad.cpu().numpy()
    rng = np.random.default_rng(1)
    checked = 0
    for s, p in zip(rng.integers(0, b.S, 60), rng.integers(0, 4096, 60)):
        a, c = b.offsets[s], b.offsets[s + 1]
        x = dls.damped_solve(dls.basis(b.omega[a:c], th[s, p]), dls.target(re[a:c], im[a:c]), dls.LAM_SEARCH)
        cref, gref = varpro.cost_grad(b.omega[a:c], re[a:c], im[a:c], th[s, p])
        assert abs(cost[s, p] - cref) <= COST_TOL[prec] * cref
        if np.min(np.abs(x[1:])) < 1e-6 * np.abs(x).max():
            continue
        assert np.linalg.norm(grad[s, p] - gref) <= GRAD_TOL[prec] * np.linalg.norm(gref), (s, p)
        checked += 1
    assert checked >= 40


def test_hn256_polish_fit_sampled(D, hn256):
    # the differentiation workload as the benchmark runs it: 4096 random candidates per
    # spectrum, the best 32 polished by 50 L-BFGS iterations (captured as a CUDA graph).
    # The starting points are the oracle's (same seeded population, same ranking); every
    # checked spectrum meets the end-to-end criterion of fitcheck (strict, or within the
    # oracle's own spread where its polish is chaotic).
    b, re, im = hn256
    with D.Handle("mixed") as h:
        out = D.debye_fit_batch(h, _spectra(D, b, re, im), P=4096, iters=0, seed=0, polish_topk=32,
                                polish_iters=50)
        D.debye_sync(h)
    how = []
    for s in (3, 77, 150):
        a, c = b.offsets[s], b.offsets[s + 1]
        e_gpu = models.multi_debye(b.omega[a:c], out["eps_inf"][s].item(), out["d_eps"][s].cpu().numpy(),
                                   out["tau"][s].cpu().numpy())
        g = out["final_cost"][s].item()
        ok, kind = fitcheck.check_spectrum(b.omega[a:c], re[a:c], im[a:c], 8, -13.0, -5.0, 4096, 0, 0, s, 32, 50,
                                           e_gpu, g)
        assert ok, (s, kind, g)
        how.append(kind)
        assert np.all(out["d_eps"][s].cpu().numpy() >= 0)
    print(how)


@pytest.mark.parametrize("prec", ["mixed", "mixed_table"])
def test_tabulated_full_size_sampled(D, prec):
    # 16384 spectra x 4096 frequencies, N = 20, 512 candidates each (mixed precision, the
    # column sums swept directly and read from the tables)
    b = W.workload("tabulated_16384_k4096")
    tt = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    om = tt(b.omega)
    offs = tt(b.offsets, torch.int64)
    with D.Handle(prec) as h:
        er, ei = D.debye_synth_targets(h, offs, om, tt(b.model, torch.int32), tt(b.params),
                                       tt(b.pole_offsets, torch.int64), tt(b.pole_tau), tt(b.pole_deps),
                                       tt(b.noise_re), tt(b.noise_im))
        sp = D.Spectra(offs, om, er, ei, tt(b.n_poles, torch.int32), tt(b.lo), tt(b.hi),
                       np.ascontiguousarray(b.offsets), np.ascontiguousarray(b.n_poles, np.int32))
        th = torch.as_tensor(W.population(b, 512, seed=0), device="cuda")
        cost = D.debye_eval_population(h, sp, th)
        D.debye_sync(h)
    cost = cost.cpu().numpy()
    th = th.cpu().numpy()
    rng = np.random.default_rng(2)
    picks = list(zip(rng.integers(0, b.S, 40), rng.integers(0, 512, 40)))
    sub = b.subset(sorted({int(s) for s, _ in picks}))
    re, im = models.synthesize(sub)
    idx = {int(s): i for i, s in enumerate(sorted({int(s) for s, _ in picks}))}
    for s, p in picks:
        i = idx[int(s)]
        a, c = sub.offsets[i], sub.offsets[i + 1]
        ref = float(dls.cost(sub.omega[a:c], re[a:c], im[a:c], th[s, p]))
        assert abs(cost[s, p] - ref) <= COST_TOL[prec] * ref, (s, p, cost[s, p], ref)


@pytest.mark.parametrize("prec,lanes", [("fp64", 0), ("mixed", 1), ("mixed", 32), ("mixed_table", 1),
                                        ("mixed_table", 32)])
def test_tabulated_cost_grad_sampled(D, prec, lanes):
    # N = 20, K = 4096 noisy Debye-sum spectra: cost and gradient of sampled candidates
    # (mixed: the small-system solve one thread and one warp per candidate)
    b = W.workload("tabulated_16384_k4096").subset(np.arange(32))
    re, im = models.synthesize(b)
    th = W.population(b, 64, seed=4)
    with D.Handle(prec, solve_lanes=lanes) as h:
        cost, grad = D.debye_cost_grad(h, _spectra(D, b, re, im), torch.as_tensor(th, device="cuda"))
        D.debye_sync(h)
    cost, grad = cost.cpu().numpy(), grad.cpu().numpy()
    rng = np.random.default_rng(5)
    checked = 0
    for s, p in zip(rng.integers(0, b.S, 16), rng.integers(0, 64, 16)):
        a, c = b.offsets[s], b.offsets[s + 1]
        x = dls.damped_solve(dls.basis(b.omega[a:c], th[s, p]), dls.target(re[a:c], im[a:c]), dls.LAM_SEARCH)
        cref, gref = varpro.cost_grad(b.omega[a:c], re[a:c], im[a:c], th[s, p])
        assert abs(cost[s, p] - cref) <= COST_TOL[prec] * cref, (s, p)
        if np.min(np.abs(x[1:])) < 1e-6 * np.abs(x).max():
            continue
        assert np.linalg.norm(grad[s, p] - gref) <= GRAD_TOL[prec] * np.linalg.norm(gref), (s, p)
        checked += 1
    assert checked >= 8
