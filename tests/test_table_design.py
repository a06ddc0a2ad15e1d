"""The column-sum tables' shape (DEBYE_PREC_MIXED_TABLE), checked in FP64 on the CPU.

Per spectrum, the pole-wise column sums S(theta) = sum_k 1/(1 + w_k^2 tau^2),
h(theta) = a(theta)^T b and their theta derivatives are interpolated on segments
of TAB_W decades by TAB_NC Chebyshev coefficients (values at the Chebyshev points
of the first kind, discrete cosine transform), stored as polynomials in the
segment's coordinate x in [-1, 1] as the kernels store them. The constants are
read from the kernel source; the interpolants, built here in numpy from exact FP64 sums, must
reproduce the direct sums to well below the float-float rounding of the GPU's
own sums (~1e-12 relative) on spectra of the benchmark workloads.
"""
import os
import re

import numpy as np

import workloads as W
from oracle import models

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LN10 = np.log(10.0)


def constants():
    text = open(os.path.join(ROOT, "paper_2109_01928_gb300", "csrc", "common.cuh")).read()
    w = float(re.search(r"constexpr double TAB_W = ([0-9.]+);", text).group(1))
    nc = int(re.search(r"constexpr int TAB_NC = (\d+);", text).group(1))
    return w, nc


def column_sums(om, er, ei, theta):
    """S, h, tau, dS/dtheta, dh/dtheta of single Debye poles at log10 tau = theta (rows),
    in the order of the tables."""
    tau = 10.0 ** np.asarray(theta)
    x = np.outer(tau, om)
    re_ = 1.0 / (1.0 + x * x)
    im_ = x * re_
    S = re_.sum(1)
    h = re_ @ er + im_ @ ei
    # d re / d theta = -2 ln10 x^2 re^2, d im / d theta = ln10 x (1 - x^2) re^2
    dre = -2.0 * LN10 * x * x * re_ * re_
    dim = LN10 * x * (1.0 - x * x) * re_ * re_
    return np.stack([S, h, tau, dre.sum(1), dre @ er + dim @ ei])


def table(om, er, ei, lo, hi, w, nc):
    nseg = max(1, int(np.ceil((hi - lo) / w)))
    m = np.arange(nc)
    xm = np.cos(np.pi * (m + 0.5) / nc)
    T = np.cos(np.pi * np.outer(np.arange(nc), m + 0.5) / nc)
    coef = []
    for g in range(nseg):
        F = column_sums(om, er, ei, lo + w * (g + 0.5 + 0.5 * xm))
        c = 2.0 / nc * F @ T.T
        c[:, 0] *= 0.5
        # stored, as on the GPU, as a polynomial in the segment's coordinate x
        coef.append(np.array([np.polynomial.chebyshev.cheb2poly(row) for row in c]))
    return np.array(coef)


def interpolate(coef, lo, w, theta):
    u = (theta - lo) / w
    g = np.minimum(u.astype(int), len(coef) - 1)
    x = 2.0 * (u - g) - 1.0
    out = np.empty((5, len(theta)))
    for i in range(len(theta)):
        out[:, i] = np.polynomial.polynomial.polyval(x[i], coef[g[i]].T)
    return out


def check_batch(b, spectra, n_theta=150):
    w, nc = constants()
    re_all, im_all = models.synthesize(b)
    rng = np.random.default_rng(11)
    worst = np.zeros(5)
    for s in spectra:
        a, c = b.offsets[s], b.offsets[s + 1]
        om, er, ei = b.omega[a:c], re_all[a:c], im_all[a:c]
        lo, hi = float(b.lo[s]), float(b.hi[s])
        coef = table(om, er, ei, lo, hi, w, nc)
        th = np.concatenate([rng.uniform(lo, hi, n_theta), [lo, hi]])
        got, ref = interpolate(coef, lo, w, th), column_sums(om, er, ei, th)
        # S, h and tau relative to themselves; the derivatives change sign: relative to their range
        scale = np.stack([np.abs(ref[0]), np.abs(ref[1]), ref[2],
                          np.full(len(th), np.abs(ref[3]).max()), np.full(len(th), np.abs(ref[4]).max())])
        worst = np.maximum(worst, (np.abs(got - ref) / scale).max(axis=1))
    return worst


def test_table_shape_mixed_workload():
    b = W.workload("mixed_1024")
    worst = check_batch(b, [0, 4, 6, 3, 1, 400])   # HN, CC, CD, Jonscher, CRIM and one more
    assert worst[:3].max() <= 1e-13 and worst[3:].max() <= 5e-13, worst


def test_table_shape_tabulated_workload():
    b = W.tabulated_batch(S=4, K=1024, seed=3)            # 40 random poles, Jonscher tail, 1 % noise
    worst = check_batch(b, range(4))
    assert worst[:3].max() <= 1e-13 and worst[3:].max() <= 5e-13, worst


def test_coarser_table_is_not_enough():
    # the bound is not slack: 8 coefficients on the same segments miss by orders of magnitude
    w, nc = constants()
    b = W.workload("mixed_1024")
    re_all, im_all = models.synthesize(b)
    a, c = b.offsets[0], b.offsets[1]
    om, er, ei = b.omega[a:c], re_all[a:c], im_all[a:c]
    coef = table(om, er, ei, float(b.lo[0]), float(b.hi[0]), w, 8)
    th = np.random.default_rng(1).uniform(b.lo[0], b.hi[0], 100)
    got, ref = interpolate(coef, float(b.lo[0]), w, th), column_sums(om, er, ei, th)
    assert (np.abs(got[0] - ref[0]) / ref[0]).max() > 1e-12
