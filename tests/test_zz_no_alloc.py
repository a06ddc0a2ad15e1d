"""The allocation-free evaluation entry point against the handle-based one.

debye_eval_population_noalloc serves callers that cannot let the library
allocate device memory (an application with a fixed device-memory budget, or a
loop where cudaMalloc's device synchronisation is not acceptable): it keeps all
temporaries in a fixed array inside the library. This file is collected last so
that a run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import models

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
# The two entry points may split candidates over different numbers of lanes (the
# handle path sizes the split to the batch), so sums run in different orders:
# weights, not stationary like the cost, are compared at the oracle-parity
# tolerance of their own scale.
WTOL = {"fp64": 1e-7, "mixed": 2e-3}


@pytest.fixture(scope="module")
def D():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2109_01928_gb300 import debyefit
    debyefit.lib()
    return debyefit


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_eval_population_twice(D, prec):
    # a ragged batch with every kernel bucket (N = 1..20), small enough for the fixed scratch
    b = W.mixed_batch(S=20, seed=13, P=24, K_range=(30, 300), N_range=(1, 20))
    b.n_poles[:] = np.arange(1, 21)
    re, im = models.synthesize(b)
    sp = D.make_spectra(b.offsets, b.omega, re, im, b.n_poles, b.lo, b.hi, device="cuda")
    with D.Handle(prec) as h:
        for call, seed in enumerate((1, 2)):   # two calls in a row, different populations
            th = torch.as_tensor(W.population(b, 24, seed=seed), device="cuda")
            ref_c, ref_w = D.debye_eval_population(h, sp, th, weights=True)
            c, w = D.debye_eval_population_noalloc(sp, th, precision=prec, weights=True)
            torch.cuda.synchronize()
            rc, rw = ref_c.cpu().numpy(), ref_w.cpu().numpy()
            err = np.abs(c.cpu().numpy() - rc) / rc
            assert err.max() <= TOL[prec], (call, err.max())
            scale = np.abs(rw).max(axis=2, keepdims=True)
            assert (np.abs(w.cpu().numpy() - rw) / scale).max() <= WTOL[prec], call


def test_noalloc_rejects_batches_beyond_the_scratch(D):
    b = W.workload("mixed_1024")
    re, im = models.synthesize(b)
    sp = D.make_spectra(b.offsets, b.omega, re, im, b.n_poles, b.lo, b.hi, device="cuda")
    th = torch.zeros((b.S, b.P, b.n_max), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DebyeError) as e:
        D.debye_eval_population_noalloc(sp, th)
    assert e.value.code == D.DEBYE_EINVAL
    assert "scratch" in str(e.value) or "work units" in str(e.value)
