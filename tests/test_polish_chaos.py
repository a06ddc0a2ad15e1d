"""The FP64 oracle's own sensitivity to 1e-9 perturbations of its polish start points.

This pins the claim behind the end-to-end criterion of fitcheck: on an
over-parameterised spectrum (a CRIM mixture whose only relaxation is the water
pole, fitted with 9 poles) the oracle's polished result moves by more than
1e-4 relative RMS and several per cent in cost when its start points move by
1e-9 decades, while on a well-posed spectrum (6 poles for a Havriliak-Negami
spectrum of the same batch) it does not move beyond rounding.
"""
import numpy as np
import pytest

import fitcheck
import workloads as W
from oracle import dls, models

pytestmark = pytest.mark.slow


def spread(s):
    b = W.workload("mixed_1024").subset([s])
    re, im = models.synthesize(b)
    runs = fitcheck.perturbed_oracle_fits(b.omega, re, im, int(b.n_poles[0]), float(b.lo[0]), float(b.hi[0]),
                                          256, 200, 0, s, 8, 50, repeats=2)
    c0, e0 = runs[0]
    return b, [(abs(c - c0) / c0, dls.rel_rms(e, e0)) for c, e in runs[1:]]


def test_polish_is_chaotic_on_an_over_parameterised_spectrum():
    b, d = spread(359)
    assert b.model[0] == W.MODEL_CRIM and b.n_poles[0] == 9
    assert max(r for _, r in d) > 1e-4 and max(c for c, _ in d) > 1e-2, d


def test_polish_is_stable_on_a_well_posed_spectrum():
    b, d = spread(0)
    assert b.n_poles[0] == 6
    assert max(r for _, r in d) < 1e-7 and max(c for c, _ in d) < 1e-10, d
