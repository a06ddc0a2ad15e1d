"""The allocation-free evaluation entry point, through the C ABI.

debye_eval_population_noalloc serves callers that cannot let the library
allocate device memory (an application with a fixed device-memory budget, or a
loop where cudaMalloc's device synchronisation is not acceptable): it keeps all
temporaries in a fixed array inside the library. Its results are checked
against the handle-based debye_eval_population and against the FP64 oracle,
on two calls in a row (the scratch keeps the previous call's contents). This
file is collected last so that a run stopping at its first failure has already
run every other test.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dls, models

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5, "mixed_table": 1e-5}
# The two entry points may split candidates over different numbers of lanes (the
# handle path sizes the split to the batch), so sums run in different orders and
# the weights, which are not stationary like the cost, differ by rounding: FP64
# weights to ~1e-12 of their scale, mixed ones to the refinement bound
# (kappa 2^-24)^2 ~ 1.6e-6 with kappa <= (n + lam) / lam (n = 21, lam = 1e-3).
WTOL = {"fp64": 1e-10, "mixed": 1e-5, "mixed_table": 1e-5}


@pytest.fixture(scope="module")
def D():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2109_01928_gb300 import debyefit
    debyefit.lib()
    return debyefit


def oracle_costs(b, re, im, th):
    out = np.empty(th.shape[:2])
    for s in range(b.S):
        a, c = b.offsets[s], b.offsets[s + 1]
        out[s] = dls.cost_population(b.omega[a:c], re[a:c], im[a:c], th[s, :, :int(b.n_poles[s])])[0]
    return out


# (population, cands_per_block option): P = 24 takes the small-population layout
# (two lanes per candidate); P = 64 one lane per candidate in 64-candidate units;
# P = 64 with cands_per_block = 128 the forced block size.
LAYOUTS = [(24, 0), (64, 0), (64, 128)]


# mixed_table: the entry point takes the direct column sums, the handle the tables
@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_table"])
@pytest.mark.parametrize("P,cb", LAYOUTS)
def test_noalloc_matches_eval_population_twice(D, prec, P, cb):
    # a ragged batch with every kernel bucket (N = 1..20), small enough for the fixed scratch
    b = W.mixed_batch(S=20, seed=13, P=P, K_range=(30, 300), N_range=(1, 20))
    b.n_poles[:] = np.arange(1, 21)
    re, im = models.synthesize(b)
    sp = D.make_spectra(b.offsets, b.omega, re, im, b.n_poles, b.lo, b.hi, device="cuda")
    opts = D.default_options()
    opts.cands_per_block = cb
    with D.Handle(prec, cands_per_block=cb) as h:
        for call, seed in enumerate((1, 2)):   # two calls in a row, different populations
            thn = W.population(b, P, seed=seed)
            th = torch.as_tensor(thn, device="cuda")
            ref_c, ref_w = D.debye_eval_population(h, sp, th, weights=True)
            c, w = D.debye_eval_population_noalloc(sp, th, precision=prec, weights=True, options=opts)
            torch.cuda.synchronize()
            rc, rw = ref_c.cpu().numpy(), ref_w.cpu().numpy()
            c, w = c.cpu().numpy(), w.cpu().numpy()
            err = np.abs(c - rc) / rc
            assert err.max() <= TOL[prec], (call, err.max())
            scale = np.abs(rw).max(axis=2, keepdims=True)
            assert (np.abs(w - rw) / scale).max() <= WTOL[prec], call
            oracle = oracle_costs(b, re, im, thn)
            assert (np.abs(c - oracle) / oracle).max() <= TOL[prec], call


def test_noalloc_rejects_batches_beyond_the_scratch(D):
    b = W.workload("mixed_1024")
    re, im = models.synthesize(b)
    sp = D.make_spectra(b.offsets, b.omega, re, im, b.n_poles, b.lo, b.hi, device="cuda")
    th = torch.zeros((b.S, b.P, b.n_max), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DebyeError) as e:
        D.debye_eval_population_noalloc(sp, th)
    assert e.value.code == D.DEBYE_EINVAL
    assert "scratch" in str(e.value) or "work units" in str(e.value)
