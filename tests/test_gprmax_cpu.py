"""The gprMax command layer (Sec. IV, Listings 1 and 2) without a GPU: parsing,
the frequency grid and search bounds, and the output format."""
import math

import numpy as np
import pytest

from paper_2109_01928_gb300 import gprmax as G

LISTING_1 = "#havriliak_negami: 1e7 1e11 0.91 0.45 2.7 5.9 9.4e-10 0.1 1 0 5 Kelley"


def test_parse_paper_listing():
    (c,) = G.parse(LISTING_1)
    assert c.kind == "havriliak_negami" and c.model == G.MODEL_HN
    assert (c.f_lo, c.f_hi) == (1e7, 1e11)
    np.testing.assert_array_equal(c.params[:5], [2.7, 5.9, 9.4e-10, 0.91, 0.45])
    assert (c.sigma, c.mu_r, c.sigma_m, c.n_poles, c.ident, c.seed) == ("0.1", "1", "0", 5, "Kelley", 0)
    (c2,) = G.parse(LISTING_1 + " 17")
    assert c2.seed == 17


def test_parse_other_commands(tmp_path):
    txt = """
    ## a comment line
    #jonscher: 1e6 1e10 4.0 5.0 6.283e8 0.6 0.01 1 0 -1 clay 3
    #crim: 1e6 1e10 0.5 2 0.3 0.7 4.9 75 9.23e-12 4.5 0 1e-12 0 1 0 6 wetsand
    #raw_data: meas.txt 0.05 1 0 4 sample
    #domain: 1 1 1
    """
    f = np.logspace(6, 9, 30)
    np.savetxt(tmp_path / "meas.txt", np.stack([f, 5 + 1 / (1 + (f / 1e8) ** 2), 0.3 * np.ones_like(f)], 1))
    cmds = G.parse(txt, str(tmp_path))
    assert [c.kind for c in cmds] == ["jonscher", "crim", "raw_data"]
    j, c, r = cmds
    np.testing.assert_array_equal(j.params[:4], [4.0, 5.0, 6.283e8, 0.6])
    assert j.n_poles == -1 and j.seed == 3
    assert c.params[0] == 0.5 and c.params[1] == 2
    np.testing.assert_array_equal(c.params[2:4], [0.3, 0.7])
    np.testing.assert_array_equal(c.params[5:11], [4.9, 75, 9.23e-12, 4.5, 0, 1e-12])
    assert c.n_poles == 6 and c.ident == "wetsand"
    assert r.model == -1 and r.data.shape == (30, 3) and (r.f_lo, r.f_hi) == (f[0], f[-1])


@pytest.mark.parametrize("bad", [
    "#havriliak_negami: 1e7 1e11 0.91 0.45 2.7 5.9 9.4e-10 0.1 1 0 21 X",
    "#havriliak_negami: 1e7 1e11 1.5 0.45 2.7 5.9 9.4e-10 0.1 1 0 5 X",
    "#havriliak_negami: 1e7 1e11 0.91 0.45 2.7",
    "#crim: 1e6 1e10 0.5 4 0.3 0.7",
    "#jonscher: 1e6 1e10 4.0 5.0 x 0.6 0.01 1 0 3 clay",
])
def test_parse_errors(bad):
    with pytest.raises(G.CommandError):
        G.parse(bad)


def test_grid_and_bounds():
    om = G.frequency_grid(1e7, 1e11)
    assert om.size == 201
    np.testing.assert_allclose(om[[0, -1]], 2 * math.pi * np.array([1e7, 1e11]), rtol=1e-15)
    assert np.all(np.diff(np.log(om)) > 0)
    # the paper example's search range [-13, -6] (relaxation frequencies 1e7-1e11 Hz with a decade of margin)
    assert G.tau_bounds(1e7, 1e11) == (-13.0, -6.0)
    assert G.frequency_grid(1e8, 1.5e8).size == 50


def test_output_format_matches_listing_2():
    (c,) = G.parse(LISTING_1)
    d = [2.3563, 0.6736, 1.1009, 1.2926, 0.3091]
    t = [4.3677e-10, 1.1623e-11, 1.5180e-9, 9.1048e-11, 1.1131e-12]
    out = G.format_result(c, 2.8345, d, t)
    assert out.splitlines()[0] == "#material: 2.8345 0.1 1 0 Kelley"
    assert out.splitlines()[1] == ("#add_dispersion_debye: 5 2.3563 4.3677e-10 0.6736 1.1623e-11 1.1009 "
                                   "1.5180e-09 1.2926 9.1048e-11 0.3091 1.1131e-12 Kelley")
