"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from a
closed form, a textbook identity, an independent library routine (SVD least
squares, normal equations, finite differences, brute-force grids) or a value
printed in the paper (tests/golden/).
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import da, de, dls, dmath, fit, lbfgs, models, pso, rng, varpro

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid(f_lo=1e6, f_hi=1e10, K=200):
    return W.log_grid(f_lo, f_hi, K)


# ---------------------------------------------------------------- targets (Eqs. 3-7)

def test_hn_alpha_beta_one_is_debye():
    om = grid(1e5, 1e11, 300)
    hn = models.havriliak_negami(om, 3.0, 12.0, 2e-10, 1.0, 1.0)
    # Debye written out in real form: eps' = ei + de/(1+x^2), eps'' = de x/(1+x^2)
    x = om * 2e-10
    np.testing.assert_allclose(hn.real, 3.0 + 12.0 / (1 + x * x), rtol=1e-15, atol=0)
    np.testing.assert_allclose(-hn.imag, 12.0 * x / (1 + x * x), rtol=1e-14, atol=0)


def test_cole_cole_at_relaxation_frequency():
    # (1 + j^alpha)^-1 = 1/2 - (j/2) tan(alpha pi / 4) at w tau0 = 1
    for alpha in (0.3, 0.55, 0.91, 1.0):
        tau0 = 3.3e-9
        e = models.cole_cole(np.array([1.0 / tau0]), 2.0, 7.0, tau0, alpha)
        assert abs(e.real[0] - (2.0 + 3.5)) < 1e-13
        assert abs(-e.imag[0] - 3.5 * math.tan(alpha * math.pi / 4)) < 1e-13


def test_cole_davidson_closed_form():
    # eps - eps_inf = d_eps cos^beta(phi) exp(-j beta phi), phi = atan(w tau0)
    om = grid(1e5, 1e11, 100)
    tau0, beta = 1.7e-9, 0.45
    e = models.cole_davidson(om, 4.0, 20.0, tau0, beta)
    phi = np.arctan(om * tau0)
    ref = 4.0 + 20.0 * np.cos(phi) ** beta * np.exp(-1j * beta * phi)
    np.testing.assert_allclose(e, ref, rtol=1e-13)


def test_hn_real_form():
    # Textbook modulus/argument form of Eq. 4
    om = grid(1e5, 1e11, 200)
    ei, de, tau0, a, b = 2.7, 5.9, 9.4e-10, 0.91, 0.45
    e = models.havriliak_negami(om, ei, de, tau0, a, b)
    wt = (om * tau0) ** a
    rr = 1 + 2 * wt * math.cos(a * math.pi / 2) + wt * wt
    th = np.arctan2(wt * math.sin(a * math.pi / 2), 1 + wt * math.cos(a * math.pi / 2))
    np.testing.assert_allclose(e.real, ei + de * rr ** (-b / 2) * np.cos(b * th), rtol=1e-14)
    np.testing.assert_allclose(-e.imag, de * rr ** (-b / 2) * np.sin(b * th), rtol=1e-13)


def test_debye_loss_peak_at_relaxation_frequency():
    # eps'' peaks at f0 = 1/(2 pi tau0) with value d_eps/2 (Sec. II-B, Fig. 1)
    tau0 = 0.1e-9
    f = np.logspace(8, 11, 30001)
    e = models.debye(2 * math.pi * f, 1.0, 14.0, tau0)
    k = np.argmax(-e.imag)
    assert abs(math.log10(f[k]) - math.log10(1 / (2 * math.pi * tau0))) < 2e-4
    assert abs(-e.imag[k] - 7.0) < 1e-6


def test_crim_special_cases():
    om = grid()
    water = W.WATER
    e1 = models.crim(om, [1.0, 0.0, 0.0], [water, W.SAND, W.AIR])
    np.testing.assert_allclose(e1, models.debye(om, *water), rtol=1e-14)
    e2 = models.crim(om, [0.3, 0.7], [W.SAND, W.AIR])
    assert np.allclose(e2, (0.3 * math.sqrt(4.5) + 0.7) ** 2, rtol=1e-14)


def test_jonscher_loss_ratio():
    om = grid(1e6, 1e10, 80)
    for n in (0.3, 0.6, 0.9):
        e = models.jonscher(om, 5.0, 3.0, W.OMEGA_P, n)
        np.testing.assert_allclose(-e.imag / (e.real - 5.0), 1 / math.tan(n * math.pi / 2), rtol=1e-12)
        e5 = models.jonscher_eq5(om, 5.0, 3.0, W.OMEGA_P, n)
        np.testing.assert_allclose(-e5.imag / (e5.real - 5.0), math.tan(n * math.pi / 2), rtol=1e-12)


def test_synthesize_dispatch_matches_model_functions():
    b = W.mixed_batch(S=40, seed=3)
    re, im = models.synthesize(b)
    for s in range(b.S):
        a, c = b.offsets[s], b.offsets[s + 1]
        p = b.params[s]
        if b.model[s] == W.MODEL_HN:
            e = models.havriliak_negami(b.omega[a:c], *p[:5])
            np.testing.assert_array_equal(re[a:c], e.real)
    assert np.all(im > 0)   # every drawn model is lossy at every frequency


# ---------------------------------------------------------------- damped LS cost (Sec. III)

def _debye_sum_target(om, ei, de, tau):
    e = models.multi_debye(om, ei, de, tau)
    return models.split(e)


def test_undamped_solve_matches_svd_lstsq():
    om = grid()
    rng_ = np.random.default_rng(0)
    re, im = models.split(models.havriliak_negami(om, 3.0, 30.0, 1e-9, 0.7, 0.6))
    for _ in range(10):
        th = np.sort(rng_.uniform(-11, -7, 4))
        A = dls.basis(om, th)
        b = dls.target(re, im)
        x = dls.damped_solve(A, b, 0.0)
        x_ref = np.linalg.lstsq(A, b, rcond=None)[0]   # SVD (gelsd)
        np.testing.assert_allclose(x, x_ref, rtol=1e-7, atol=1e-9 * np.abs(x_ref).max())


def test_damped_cost_is_min_of_augmented_system():
    # min_x ||A x - b||^2 + lam ||D x||^2 = squared residual of [A; sqrt(lam) D] x ~ [b; 0],
    # solved independently by SVD least squares
    om = grid(1e6, 1e10, 120)
    re, im = models.split(models.havriliak_negami(om, 4.0, 50.0, 3e-10, 0.5, 0.8))
    rng_ = np.random.default_rng(1)
    for lam in (1e-3, 1e-5, 1e-1):
        for _ in range(8):
            th = rng_.uniform(-12, -6, 5)
            A = dls.basis(om, th)
            b = dls.target(re, im)
            D = np.diag(np.linalg.norm(A, axis=0))
            aug = np.vstack([A, math.sqrt(lam) * D])
            xs, *_ = np.linalg.lstsq(aug, np.concatenate([b, np.zeros(A.shape[1])]), rcond=None)
            ref_min = float(np.sum((aug @ xs - np.concatenate([b, np.zeros(A.shape[1])])) ** 2))
            x = dls.damped_solve(A, b, lam)
            if np.all(x[1:] >= 0):
                assert abs(dls.cost(om, re, im, th, lam) - ref_min) <= 1e-10 * ref_min
            np.testing.assert_allclose(x, xs, rtol=1e-8, atol=1e-10 * np.abs(xs).max())


def test_damped_solve_matches_normal_equations():
    om = grid(1e6, 1e10, 300)
    re, im = models.split(models.cole_cole(om, 3.0, 20.0, 1e-9, 0.8))
    th = np.array([-10.5, -9.0, -7.5])
    A = dls.basis(om, th)
    b = dls.target(re, im)
    G = A.T @ A
    lam = 1e-3
    assert np.linalg.cond(G) < 1e4
    x_ne = np.linalg.solve(G + lam * np.diag(np.diag(G)), A.T @ b)
    np.testing.assert_allclose(dls.damped_solve(A, b, lam), x_ne, rtol=1e-10)


def test_exact_recovery_of_debye_sum():
    om = grid(1e6, 1e10, 400)
    tau = np.array([3e-11, 4e-10, 6e-9])
    de = np.array([5.0, 12.0, 30.0])
    re, im = _debye_sum_target(om, 2.5, de, tau)
    c, w = dls.cost(om, re, im, np.log10(tau), 0.0, return_weights=True)
    b = dls.target(re, im)
    assert c <= 1e-20 * float(b @ b)
    np.testing.assert_allclose(w, np.concatenate([[2.5], de]), rtol=1e-9)


def test_fitter_recovers_an_exact_debye_sum():
    # with (almost) no damping the search + polish finds the generating poles of
    # an exact two-pole Debye sum: tau to 1e-6 decades, the weights to 1e-6
    om = grid(1e6, 1e11, 150)
    tau = np.array([2e-11, 3e-9])
    d_eps = np.array([15.0, 40.0])
    re, im = _debye_sum_target(om, 3.0, d_eps, tau)
    r = fit.fit_spectrum(om, re, im, 2, -13.0, -6.0, 32, 40, topk=4, polish_iters=60,
                         lam_search=1e-12, lam_final=0.0)
    assert np.max(np.abs(np.log10(r["tau"]) - np.log10(tau))) <= 1e-6
    assert np.all(r["d_eps"] >= 0)
    np.testing.assert_allclose(r["d_eps"], d_eps, rtol=1e-6)
    assert abs(r["eps_inf"] - 3.0) <= 1e-6 * 3.0


def test_flip_keeps_eps_inf_sign():
    # eps_inf < 0 is not a 'negative weight' of a Debye pole: no penalty
    om = grid(1e6, 1e10, 200)
    tau = np.array([1e-10, 1e-8])
    re, im = _debye_sum_target(om, -1.0, np.array([4.0, 9.0]), tau)
    c = dls.cost(om, re, im, np.log10(tau), 0.0)
    assert c <= 1e-20 * float(re @ re + im @ im)


def test_flip_penalises_negative_weight():
    # target with a negative pole: the flipped misfit must equal the misfit of |x|
    om = grid(1e6, 1e10, 200)
    tau = np.array([1e-10, 1e-8])
    re, im = _debye_sum_target(om, 3.0, np.array([4.0, -2.0]), tau)
    b = dls.target(re, im)
    c = dls.cost(om, re, im, np.log10(tau), 0.0)
    A = dls.basis(om, np.log10(tau))
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    assert x_ls[2] < 0
    xa = np.array([x_ls[0], abs(x_ls[1]), abs(x_ls[2])])
    assert abs(c - float(np.sum((A @ xa - b) ** 2))) <= 1e-9 * c
    # the penalty is 4 x_2^2 ||a_2||^2 (the flipped column's contribution)
    assert abs(c - 4 * x_ls[2] ** 2 * float(A[:, 2] @ A[:, 2])) <= 1e-7 * c


def test_cost_invariances():
    om = grid(1e6, 1e10, 150)
    re, im = models.split(models.havriliak_negami(om, 3.0, 25.0, 5e-10, 0.6, 0.7))
    th = np.array([-10.2, -9.1, -8.3, -7.0])
    c0 = dls.cost(om, re, im, th, 1e-3)
    # scaling b by s scales the cost by s^2
    assert abs(dls.cost(om, 3 * re, 3 * im, th, 1e-3) - 9 * c0) <= 1e-11 * 9 * c0
    # permuting the poles leaves the cost unchanged
    assert abs(dls.cost(om, re, im, th[::-1], 1e-3) - c0) <= 1e-11 * c0
    # w -> c w with tau -> tau / c leaves the cost unchanged
    assert abs(dls.cost(om * 100.0, re, im, th - 2.0, 1e-3) - c0) <= 1e-9 * c0


# ---------------------------------------------------------------- gradient (VarPro)

@pytest.mark.parametrize("lam", [1e-3, 1e-6])
def test_gradient_matches_central_differences(lam):
    om = grid(1e6, 1e10, 200)
    re, im = models.split(models.havriliak_negami(om, 3.0, 25.0, 5e-10, 0.6, 0.7))
    rng_ = np.random.default_rng(5)
    n_flip = 0
    for _ in range(20):
        th = rng_.uniform(-12, -6, 4)
        x = dls.damped_solve(dls.basis(om, th), dls.target(re, im), lam)
        if np.min(np.abs(x[1:])) < 1e-8:
            continue
        n_flip += bool(np.any(x[1:] < 0))
        c, g = varpro.cost_grad(om, re, im, th, lam)
        h = 1e-6
        fd = np.array([(dls.cost(om, re, im, th + h * e, lam) - dls.cost(om, re, im, th - h * e, lam))
                       / (2 * h) for e in np.eye(4)])
        assert np.max(np.abs(g - fd)) <= 1e-6 * max(1.0, np.max(np.abs(fd))) + 1e-6 * c
    assert n_flip > 0   # the penalised branch was exercised


def test_gradient_envelope_form_without_flip():
    # with no weight flipped the weights minimise the damped cost, so its total
    # derivative equals the partial derivative at fixed weights (envelope theorem):
    # d/d theta_i [||A x - b||^2 + lam sum_j G_jj x_j^2] with x held at x*(theta),
    # here by central differences of the basis alone
    om = grid(1e6, 1e10, 250)
    re, im = models.split(models.havriliak_negami(om, 3.0, 25.0, 5e-10, 0.6, 0.7))
    b = dls.target(re, im)
    rng_ = np.random.default_rng(8)
    checked = 0
    for _ in range(40):
        th = np.sort(rng_.uniform(-11.5, -7.5, 3))
        x = dls.damped_solve(dls.basis(om, th), b, 1e-3)
        if np.min(x[1:]) <= 1e-6 * np.abs(x).max():
            continue
        _, g = varpro.cost_grad(om, re, im, th, 1e-3)
        h = 1e-6
        env = np.array([(dls.cost_at(dls.basis(om, th + h * e), b, x, 1e-3)
                         - dls.cost_at(dls.basis(om, th - h * e), b, x, 1e-3)) / (2 * h) for e in np.eye(3)])
        assert np.max(np.abs(g - env)) <= 1e-6 * max(1.0, np.max(np.abs(env))), (th, g, env)
        checked += 1
    assert checked >= 5


def test_gradient_zero_at_exact_fit():
    om = grid(1e6, 1e10, 300)
    tau = np.array([2e-10, 5e-9])
    re, im = _debye_sum_target(om, 2.0, np.array([6.0, 10.0]), tau)
    c, g = varpro.cost_grad(om, re, im, np.log10(tau), 0.0)
    assert c < 1e-18 and np.max(np.abs(g)) < 1e-7


# ---------------------------------------------------------------- random numbers

def test_splitmix64_reference_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    state = 0
    for v in vals:
        assert rng.mix(state) == v   # mix(state) = output of a generator at 'state'
        state = (state + 0x9E3779B97F4A7C15) & rng.MASK


def test_uniform_array_matches_scalar():
    u = rng.uniform_array(7, rng.TAG_R1, 3, 11, 5, 4)
    for p in range(5):
        for d in range(4):
            assert u[p, d] == rng.uniform(7, rng.TAG_R1, 3, 11, p, d)
    big = rng.uniform_array(0, 1, 0, 0, 1000, 20)
    assert 0.0 <= big.min() and big.max() < 1.0 and abs(big.mean() - 0.5) < 0.01


def test_below_bounds_and_uniformity():
    # multiply-shift of the upper 32 bits: the extreme keys map to the ends of [0, m)
    assert rng.below(0, 7) == 0 and rng.below(rng.MASK, 7) == 6
    assert rng.below((1 << 63), 2) == 1 and rng.below((1 << 63) - 1, 2) == 0
    z = rng.key_array(3, rng.TAG_DE_IDX, 0, 0, 20000, 1)[:, 0]
    r = ((z >> np.uint64(32)) * np.uint64(7)) >> np.uint64(32)
    counts = np.bincount(r.astype(np.int64), minlength=7)
    chi2 = float(np.sum((counts - 20000 / 7) ** 2 / (20000 / 7)))
    assert counts.size == 7 and chi2 < 22.5   # 99.9 % quantile of chi-square with 6 dof


# ---------------------------------------------------------------- search

def test_de_donors_are_distinct_uniform_and_rank_mapped():
    for P in (4, 5, 17, 64):
        for g in range(1, 6):
            d = de.donors(11, 2, g, P, 3)
            assert d.min() >= 0 and d.max() < P
            for p in range(P):
                assert len({p, *d[p]}) == 4
    # brute force on a tiny population: slot j takes the r-th free index in ascending order
    P = 6
    z = rng.key_array(5, rng.TAG_DE_IDX, 1, 3, P, 3)
    d = de.donors(5, 1, 3, P, 3)
    for p in range(P):
        taken = [p]
        for j in range(3):
            free = [i for i in range(P) if i not in taken]
            r = rng.below(int(z[p, j]), P - 1 - j)
            assert d[p, j] == free[r]
            taken.append(free[r])
    # each other member is an equally likely first donor
    counts = np.zeros(8)
    for g in range(1, 801):
        counts += np.bincount(de.donors(0, 0, g, 8, 3)[:, 0], minlength=8)
    expected = 800 * 8 / 8
    assert float(np.sum((counts - expected) ** 2 / expected)) < 24.3   # 99.9 % of chi-square, 7 dof


def test_de_trial_structure():
    rs = np.random.default_rng(4)
    x = rs.uniform(-12, -6, size=(5, 3))
    # F = 0, CR = 1: every trial is another member of the population (the first donor)
    u = de.trials(x, 0, 0, 0, 1, -13.0, -5.0, f_lo=0.0, f_hi=0.0, cr=1.0)
    for p in range(5):
        assert any(np.array_equal(u[p], x[i]) for i in range(5) if i != p)
    # F = 1, CR = 1, inside the box: trial = one member plus the difference of two others
    u = de.trials(x, 0, 0, 0, 2, -40.0, 30.0, f_lo=1.0, f_hi=1.0, cr=1.0)
    for p in range(5):
        found = [(a, b, c) for a in range(5) for b in range(5) for c in range(5)
                 if len({p, a, b, c}) == 4 and np.allclose(u[p], x[a] + (x[b] - x[c]), rtol=0, atol=1e-12)]
        assert found, p
    # best/1: trial = best member plus the difference of two members other than the target
    u = de.trials(x, 3, 0, 0, 2, -40.0, 30.0, f_lo=1.0, f_hi=1.0, cr=1.0, strategy=de.BEST1)
    for p in range(5):
        assert any(len({p, b, c}) == 3 and np.allclose(u[p], x[3] + (x[b] - x[c]), rtol=0, atol=1e-12)
                   for b in range(5) for c in range(5))
    # CR = 0: exactly one coordinate comes from the mutant
    x = rs.uniform(-12, -6, size=(64, 6))
    u = de.trials(x, 0, 0, 0, 1, -13.0, -5.0, cr=0.0)
    assert np.all(np.sum(u != x, axis=1) == 1)
    # large F: every coordinate stays in the box (mutants outside are re-drawn)
    u = de.trials(x, 0, 0, 0, 1, -13.0, -5.0, f_lo=8.0, f_hi=8.0, cr=1.0)
    assert u.min() >= -13.0 and u.max() <= -5.0


@pytest.mark.parametrize("strategy", [de.RAND1, de.BEST1])
def test_de_finds_quadratic_minimum(strategy):
    target = np.array([-9.3, -7.7, -11.1])
    def f(th):
        return np.sum((th - target) ** 2, axis=1)
    x, c, gi, trace = de.de(f, 3, -13, -5, 32, 300, seed=1, strategy=strategy)
    assert np.all(np.diff(trace) <= 0)
    np.testing.assert_allclose(x[gi], target, atol=1e-4)
    assert np.all(c >= c[gi]) and np.all(c == f(x))


# ---------------------------------------------------------------- fixed-operation elementary functions

def test_dmath_log_exp_against_libm():
    rs = np.random.default_rng(0)
    x = np.concatenate([np.exp(rs.uniform(-700, 700, 20000)), rs.uniform(0.5, 2.0, 20000),
                        [1.0, 2.0, 0.5, 1e-300, 1.7e308]])
    ref = np.array([math.log(v) for v in x])
    got = dmath.log(x)
    assert np.max(np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), 1e-300))) <= 3.0
    assert dmath.log(1.0) == 0.0
    y = np.concatenate([rs.uniform(-700, 700, 20000), rs.uniform(-1, 1, 20000), [0.0, 1.0, -1.0]])
    ref = np.array([math.exp(v) for v in y])
    got = dmath.exp(y)
    assert np.max(np.abs(got - ref) / np.spacing(ref)) <= 2.0
    assert dmath.exp(0.0) == 1.0 and dmath.exp(800.0) == math.inf and dmath.exp(-800.0) == 0.0


def test_dmath_polar_gaussian():
    us = [rng.uniform_array(1, 99, 0, t, 50000, 1)[:, 0] for t in range(dmath.POLAR_TRIES)]
    vs = [rng.uniform_array(2, 99, 0, t, 50000, 1)[:, 0] for t in range(dmath.POLAR_TRIES)]
    z1, z2 = dmath.gauss_pair(us, vs)
    for z in (z1, z2):
        assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.02
        assert abs(np.mean(z ** 4) - 3.0) < 0.1            # normal kurtosis
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 0.02
    # the pair comes from the first accepted try: u^2 + v^2 = s and z1^2 + z2^2 = -2 log s
    u, v = 2 * us[0] - 1, 2 * vs[0] - 1
    s = u * u + v * v
    ok = (s > 0) & (s < 1)
    np.testing.assert_allclose((z1 ** 2 + z2 ** 2)[ok], -2 * np.log(s[ok]), rtol=1e-12)


# ---------------------------------------------------------------- dual annealing

def test_da_temperature_schedule():
    assert da.visiting_temperature(1) == da.T0
    ts = [da.visiting_temperature(t) for t in range(1, 1001)]
    assert all(a > b for a, b in zip(ts, ts[1:]))
    for t in (2, 10, 500, 1000):
        ref = da.T0 * (2 ** (da.QV - 1) - 1) / ((1 + t) ** (da.QV - 1) - 1)
        assert abs(da.visiting_temperature(t) / ref - 1) < 1e-13
    # no chain reaches the re-annealing threshold within the iteration cap
    assert ts[-1] > 2e-5 * da.T0


def test_da_visiting_scale_against_its_factors():
    qv = da.QV
    for T in (0.37, 5.0, 5230.0):
        f1 = T ** (1 / (qv - 1))
        f2 = (qv - 1) ** (4 - qv)
        f3 = 2 ** ((2 - qv) / (qv - 1))
        f4 = math.sqrt(math.pi) * f1 * f2 / (f3 * (3 - qv))
        a = 1 / (qv - 1) - 0.5
        f6 = math.pi * (1 - a) / math.sin(math.pi * (1 - a)) / math.gamma(2 - a)
        ref = (f6 / f4) ** (-(qv - 1) / (3 - qv))
        assert abs(da.sigma(T) / ref - 1) < 1e-12


def test_da_visiting_deviates_follow_the_ratio_distribution():
    # dx = sigma z1 / |z2|^a: P(dx <= v) = E_z2[Phi(v |z2|^a / sigma)], integrated numerically
    from scipy import integrate, stats
    T = 3.0
    sig = da.sigma(T)
    a = (da.QV - 1) / (3 - da.QV)
    z1, z2 = da.gauss_pairs(7, 0, 1, 20000, 0, [0, 1, 2])
    dx = da.visit(z1, z2, sig).ravel()
    for q in (0.05, 0.25, 0.5, 0.75, 0.95):
        v = float(np.quantile(dx, q))
        ref = integrate.quad(lambda y: stats.norm.cdf(v * abs(y) ** a / sig) * stats.norm.pdf(y),
                             -np.inf, np.inf)[0]
        assert abs(ref - q) < 0.01, (q, v, ref)


def test_da_wrap_and_acceptance():
    x = np.array([-13.0, -9.0, -5.0, -4.0, -14.5, 3.0])
    w = da.wrap(x, -13.0, -5.0)
    np.testing.assert_array_equal(w[:3], x[:3])
    assert np.all((w >= -13.0) & (w <= -5.0))
    np.testing.assert_allclose(w[3:], [-12.0, -6.5, -13.0], atol=1e-12)
    # generalized Metropolis: (1 - (1-qa) dE/T)^(1/(1-qa)), zero once the bracket is not positive
    T = 2.0
    for de_ in (0.0, 0.01, 0.1, 0.3):
        ref = (1 - (1 - da.QA) * de_ / T) ** (1 / (1 - da.QA))
        assert abs(float(da.accept_probability(np.array([de_]), T)[0]) - ref) < 1e-14
    assert float(da.accept_probability(np.array([T / (1 - da.QA)]), T)[0]) == 0.0
    assert float(da.accept_probability(np.array([1.0]), T)[0]) == 0.0


def test_da_finds_quadratic_minimum():
    target = np.array([-9.3, -7.7])
    def f(th):
        return np.sum((th - target) ** 2, axis=1)
    x, c, gi, trace = da.da(f, 2, -13, -5, 32, 200, seed=1)
    assert np.all(np.diff(trace) <= 0)
    np.testing.assert_allclose(x[gi], target, atol=2e-2)
    assert np.all(c == f(x))


def test_pso_finds_quadratic_minimum():
    target = np.array([-9.3, -7.7])
    def f(th):
        return np.sum((th - target) ** 2, axis=1)
    pbx, pbc, gi, trace = pso.pso(f, 2, -13, -5, 32, 200, seed=1)
    assert np.all(np.diff(trace) <= 0)
    np.testing.assert_allclose(pbx[gi], target, atol=1e-4)


def _recording(f):
    """cost function that also records every population it evaluates"""
    seen = []

    def g(th):
        seen.append((th.copy(), f(th)))
        return seen[-1][1]
    return g, seen


def test_pso_initial_state_distribution():
    # positions U[lo, hi], velocities U[-(hi - lo), hi - lo]: the first generation's
    # positions x1 = clip(x0 + v1) with omega = 1, phi = 0 give v1 = v0 = x1 - x0 where
    # unclipped; Kolmogorov-Smirnov against the two uniform laws (10^4 draws each)
    from scipy import stats
    lo, hi = -13.0, -5.0
    f, seen = _recording(lambda th: np.zeros(th.shape[0]))
    pso.pso(f, 4, lo, hi, 2500, 1, seed=3, omega=1.0, phi_p=0.0, phi_g=0.0)
    x0, x1 = seen[0][0], seen[1][0]
    assert stats.kstest(((x0 - lo) / (hi - lo)).ravel(), "uniform").pvalue > 1e-3
    free = (x1 > lo) & (x1 < hi)
    v = (x1 - x0)[free] / (hi - lo)
    # v0 ~ U[-1, 1] conditioned on x0 + v0 staying inside: compare with the same
    # conditioning applied to exact uniform draws
    rs = np.random.default_rng(0)
    u0 = rs.uniform(0, 1, 200000)
    w0 = rs.uniform(-1, 1, 200000)
    keep = (u0 + w0 > 0) & (u0 + w0 < 1)
    assert stats.ks_2samp(v, w0[keep]).pvalue > 1e-3
    assert abs(np.mean(free) - np.mean(keep)) < 0.02


def test_pso_social_term_pulls_towards_the_global_best():
    # omega = 0, phi_p = 0, phi_g = 1: v1 = r2 (g - x0) with r2 in [0, 1), so every
    # particle lands on the segment from its start to the global best of generation 0
    target = np.array([-9.0, -7.0, -11.0])
    def f(th):
        return np.sum((th - target) ** 2, axis=1)
    rec, seen = _recording(f)
    pso.pso(rec, 3, -13.0, -5.0, 64, 1, seed=5, omega=0.0, phi_p=0.0, phi_g=1.0)
    (x0, c0), (x1, _) = seen[0], seen[1]
    g = x0[int(np.argmin(c0))]
    t = (x1 - x0) / np.where(g - x0 == 0, 1.0, g - x0)
    assert np.all((t >= 0) & (t < 1) | (g - x0 == 0))
    # and not towards the particle's own start (phi_p = 1, phi_g = 0: at generation 1
    # the personal best is the start itself, so nothing moves)
    rec2, seen2 = _recording(f)
    pso.pso(rec2, 3, -13.0, -5.0, 64, 1, seed=5, omega=0.0, phi_p=1.0, phi_g=0.0)
    np.testing.assert_array_equal(seen2[1][0], seen2[0][0])


def test_pso_inertia_and_clipping():
    # omega = 1, phi = 0: straight lines with the initial velocity, clipped to the box;
    # a particle stays at a bound while its velocity points outwards
    rec, seen = _recording(lambda th: np.zeros(th.shape[0]))
    pso.pso(rec, 2, -13.0, -5.0, 50, 6, seed=7, omega=1.0, phi_p=0.0, phi_g=0.0)
    xs = np.array([x for x, _ in seen])
    assert xs.min() >= -13.0 and xs.max() <= -5.0
    v0 = xs[1] - xs[0]
    for k in range(1, len(xs)):
        expect = np.clip(xs[0] + k * v0, -13.0, -5.0)   # exact where no clip happened before
        inside = np.all([(xs[0] + j * v0 > -13.0) & (xs[0] + j * v0 < -5.0) for j in range(1, k)], axis=0) \
            if k > 1 else np.ones_like(v0, bool)
        np.testing.assert_allclose(xs[k][inside], expect[inside], rtol=0, atol=1e-12)
    assert np.any(xs == -13.0) and np.any(xs == -5.0)


def test_pso_trace_is_running_minimum_of_all_costs():
    # synchronous update, personal best replaced only on a strictly lower cost: the
    # global best after each generation is the lowest cost evaluated so far, and each
    # personal best is the lowest cost its particle has seen
    rs = np.random.default_rng(4)
    A = rs.standard_normal((3, 3))
    def f(th):
        d = th + 9.0
        return np.einsum("pi,ij,pj->p", d, A @ A.T, d) + np.sin(5 * th).sum(axis=1)
    rec, seen = _recording(f)
    pbx, pbc, gi, trace = pso.pso(rec, 3, -13.0, -5.0, 40, 30, seed=2)
    costs = np.array([c for _, c in seen])
    np.testing.assert_array_equal(trace, np.minimum.accumulate(costs.min(axis=1)))
    np.testing.assert_array_equal(pbc, costs.min(axis=0))
    assert pbc[gi] == costs.min()


def test_lbfgs_box_quadratic_and_bound():
    Q = np.array([[3.0, 1.0], [1.0, 2.0]])
    c = np.array([-9.0, -8.0])
    def fg(t):
        d = t - c
        return float(d @ Q @ d), 2 * Q @ d
    th, f, _ = lbfgs.polish(fg, np.array([-12.0, -12.0]), -13, -5, iters=100)
    np.testing.assert_allclose(th, c, atol=1e-6)
    # minimiser outside the box: lands on the bound
    th2, _, _ = lbfgs.polish(lambda t: (float((t + 4.0) @ (t + 4.0)), 2 * (t + 4.0)),
                             np.array([-12.0, -10.0]), -13, -5, iters=100)
    np.testing.assert_allclose(th2, [-5.0, -5.0], atol=1e-9)


def _brute_force_n1(om, re, im, lam):
    from scipy.optimize import minimize_scalar
    th = np.linspace(-13, -6, 7001)
    c, _ = dls.cost_population(om, re, im, th[:, None], lam, chunk=2048)
    k = int(np.argmin(c))
    res = minimize_scalar(lambda t: float(dls.cost(om, re, im, np.array([t]), lam)),
                          bracket=(th[max(k - 1, 0)], th[k], th[min(k + 1, 7000)]),
                          method="golden", tol=1e-10)
    return min(float(res.fun), float(c[k]))


def _brute_force_n2(om, re, im, lam, n=301):
    from scipy.optimize import minimize
    t = np.linspace(-13, -6, n)
    a, b = np.meshgrid(t, t, indexing="ij")
    m = a <= b
    cand = np.stack([a[m], b[m]], axis=1)
    c, _ = dls.cost_population(om, re, im, cand, lam, chunk=4096)
    best = float(np.min(c))
    for k in np.argsort(c)[:5]:
        res = minimize(lambda x: float(dls.cost(om, re, im, x, lam)), cand[k], method="Nelder-Mead",
                       options={"xatol": 1e-9, "fatol": 1e-14, "maxiter": 4000})
        best = min(best, float(res.fun))
    return best


@pytest.mark.parametrize("method", ["pso", "de", "da"])
@pytest.mark.parametrize("N", [1, 2])
def test_search_reaches_brute_force_minimum(N, method):
    b = W.single_hn(K=50, N=N)
    re, im = models.synthesize(b)
    lam = dls.LAM_SEARCH
    bf = _brute_force_n1(b.omega, re, im, lam) if N == 1 else _brute_force_n2(b.omega, re, im, lam)
    iters = 30 if method == "da" else 100
    r = fit.fit_spectrum(b.omega, re, im, N, -13.0, -6.0, 64, iters, topk=8, method=method)
    assert r["cost_search"] <= (1 + 1e-6) * bf


def _debye_target(om, eps_inf, d_eps, tau):
    e = models.multi_debye(om, eps_inf, np.asarray(d_eps, float), np.asarray(tau, float))
    return e.real.copy(), -e.imag.copy()


def test_auto_pole_count_on_exact_debye_sums():
    # a single Debye pole is recovered with N = 1; the Marquardt damping (1e-3)
    # biases the weights by well under 1 %, far below the 5 % threshold
    om = W.log_grid(1e6, 1e11, 120)
    re, im = _debye_target(om, 3.0, [20.0], [1e-9])
    r = fit.fit_auto(om, re, im, -13.0, -5.0, 32, 30, topk=4, polish_iters=30, n_hi=6)
    assert r["N"] == 1 and r["avg_frac_err"] < 1.0
    # two poles four decades apart: one pole cannot follow both loss peaks (its
    # error is far above 5 %); two poles recover the sum up to the damping bias
    re, im = _debye_target(om, 3.0, [20.0, 20.0], [1e-11, 1e-7])
    one = fit.fit_spectrum(om, re, im, 1, -13.0, -5.0, 32, 30, topk=4, polish_iters=30)
    assert one["avg_frac_err"] > 20.0
    r = fit.fit_auto(om, re, im, -13.0, -5.0, 32, 40, topk=4, polish_iters=40, n_hi=6)
    assert r["N"] == 2 and r["avg_frac_err"] < 1.0
    np.testing.assert_allclose(r["tau"], [1e-11, 1e-7], rtol=2e-2)
    # a threshold nothing reaches runs up to the cap
    r = fit.fit_auto(om, re, im, -13.0, -5.0, 16, 5, topk=0, polish_iters=0, n_hi=3, threshold=0.0)
    assert r["N"] == 3


def test_fit_is_passive_and_sorted():
    b = W.single_hn()
    re, im = models.synthesize(b)
    r = fit.fit_spectrum(b.omega, re, im, 3, -13.0, -6.0, 64, 60, topk=4)
    assert np.all(r["d_eps"] >= 0) and np.all(np.diff(r["tau"]) >= 0)
    om = W.log_grid(1e6, 1e12, 2000)
    e = fit.fitted_eps(om, r)
    assert np.all(-e.imag >= 0) and np.all(np.diff(e.real) <= 1e-12)


# ---------------------------------------------------------------- the paper's worked example

def _listing2():
    ei, poles = None, []
    for line in open(os.path.join(GOLDEN, "paper_listing2.txt")):
        if line.startswith("eps_inf"):
            ei = float(line.split()[1])
        elif line.startswith("pole"):
            poles.append((float(line.split()[1]), float(line.split()[2])))
    return ei, np.array(poles)


def test_paper_example_weights_at_printed_tau():
    ei, poles = _listing2()
    pe = W.paper_example(K=1000)
    re, im = models.synthesize(pe)
    c, w = dls.cost(pe.omega, re, im, np.log10(poles[:, 1]), 0.0, return_weights=True)
    assert abs(w[0] - ei) / ei < 0.01
    assert np.max(np.abs(w[1:] - poles[:, 0]) / poles[:, 0]) < 0.01


def test_paper_example_fit_beats_printed_result():
    ei, poles = _listing2()
    pe = W.paper_example(K=200)
    re, im = models.synthesize(pe)
    lam = dls.LAM_SEARCH
    printed = float(dls.cost(pe.omega, re, im, np.log10(poles[:, 1]), lam))
    r = fit.fit_spectrum(pe.omega, re, im, 5, -13.0, -6.0, 64, 100, topk=8)
    assert r["cost_search"] <= printed
    # Sec. IV: the PSO-DLS fit of this example stays below 10 % average fractional error
    assert r["avg_frac_err"] < 10.0
