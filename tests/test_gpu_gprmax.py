"""The gprMax command layer on the GPU: the paper's Listing 1 command fitted end to
end (targets synthesised on the device, batch fit, Listing 2 output), checked
against the oracle's fit of the same spectrum, and the automatic pole count."""
import numpy as np
import pytest

from oracle import dls, fit, models
from paper_2109_01928_gb300 import gprmax as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LISTING_1 = "#havriliak_negami: 1e7 1e11 0.91 0.45 2.7 5.9 9.4e-10 0.1 1 0 5 Kelley"


def _hn_target(om):
    e = models.havriliak_negami(om, 2.7, 5.9, 9.4e-10, 0.91, 0.45)
    return e.real.copy(), -e.imag.copy()


def test_listing_1_end_to_end_matches_oracle():
    assert torch.cuda.is_available()
    out = G.translate(LISTING_1, precision="fp64")
    l1, l2 = out.splitlines()
    assert l1.startswith("#material: ") and l1.endswith(" 0.1 1 0 Kelley")
    tok = l2.split()
    assert tok[0] == "#add_dispersion_debye:" and tok[1] == "5" and tok[-1] == "Kelley" and len(tok) == 13
    eps_inf = float(l1.split()[1])
    d_eps = np.array([float(v) for v in tok[2:12:2]])
    tau = np.array([float(v) for v in tok[3:12:2]])
    assert np.all(d_eps >= 0) and np.all(np.diff(tau) >= 0)
    om = G.frequency_grid(1e7, 1e11)
    re, im = _hn_target(om)
    r = fit.fit_spectrum(om, re, im, 5, -13.0, -6.0, 64, 100, seed=0, spectrum=0, topk=8, polish_iters=50)
    e_cmd = models.multi_debye(om, eps_inf, d_eps, tau)
    # the printed values carry 5 significant digits
    assert dls.rel_rms(e_cmd, fit.fitted_eps(om, r)) <= 1e-3
    # the paper's 10 % level for the average fractional error of this example (Sec. IV)
    err = dls.avg_fractional_error(om, re, im, np.concatenate([[eps_inf], d_eps]), np.log10(tau))
    assert err < 10.0


def test_automatic_pole_count_command():
    cmd = LISTING_1.replace(" 5 Kelley", " -1 Kelley")
    (c,) = G.parse(cmd)
    (res,) = G.fit_commands([c], precision="mixed")
    assert 1 <= res["N"] <= 20 and res["frac_err"] < 5.0
    om = G.frequency_grid(1e7, 1e11)
    re, im = _hn_target(om)
    w = np.concatenate([[res["eps_inf"]], res["d_eps"]])
    ref = dls.avg_fractional_error(om, re, im, w, np.log10(res["tau"]))
    assert abs(res["frac_err"] - ref) <= 1e-9 * ref
    # the sequential procedure stops at the first N below 5 %: a fit with N - 1 poles is
    # not good enough (a separate batch: summation order may differ, so allow 10 %)
    if res["N"] > 1:
        (c1,) = G.parse(LISTING_1.replace(" 5 Kelley", f" {res['N'] - 1} Kelley"))
        (r1,) = G.fit_commands([c1], precision="mixed")
        w1 = np.concatenate([[r1["eps_inf"]], r1["d_eps"]])
        assert dls.avg_fractional_error(om, re, im, w1, np.log10(r1["tau"])) >= 4.5
