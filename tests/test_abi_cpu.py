"""The C-ABI library without a GPU: it loads, exports every declared symbol, and
its ctypes structure layouts agree with a C compiler's view of the header."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2109_01928_gb300 import _build
from paper_2109_01928_gb300 import debyefit as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(D.LIB_PATH):
        _build.build()
    return D.lib()


def test_exports_every_declared_function(lib):
    names = D.header_functions()
    assert {"debye_fit_init", "debye_eval_population", "debye_fit_batch", "debye_cost_grad",
            "debye_sync", "debye_synth_targets", "debye_last_error"} <= set(names)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/debyefit.h but not exported"


def header_defines(prefix):
    import re
    text = open(os.path.join(ROOT, "include", "debyefit.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (" + prefix + r"\w+)\s+(-?\d+)", text)}


def test_binding_constants_match_header():
    prec = header_defines("DEBYE_PREC_")
    assert prec == {"DEBYE_PREC_" + k.upper(): v for k, v in D.PRECISIONS.items()}
    kinds = header_defines("DEBYE_KERNEL_")
    n = kinds.pop("DEBYE_KERNEL_KINDS")
    assert kinds == {"DEBYE_KERNEL_" + k.upper(): v for k, v in D.KERNEL_KINDS.items()}
    assert sorted(kinds.values()) == list(range(n))


def test_default_options(lib):
    o = D.default_options()
    assert o.precision == D.PREC_MIXED and o.refine_steps == 1
    assert o.lam_search == 1e-3 and o.lam_final == 1e-3
    assert (o.pso_omega, o.pso_phi_p, o.pso_phi_g) == (0.5, 0.5, 0.5)
    assert o.lbfgs_m == 8 and o.lbfgs_max_trials == 20 and o.lbfgs_c1 == 1e-4
    assert (o.de_f_lo, o.de_f_hi, o.de_cr, o.de_strategy) == (0.5, 1.0, 0.7, D.DE_RAND1)
    assert (o.da_t0, o.da_qa) == (5230.0, -5.0)
    assert o.solve_lanes == 0


def test_init_rejects_bad_options(lib):
    o = D.default_options()
    o.refine_steps = 0
    h = ctypes.c_void_p()
    assert lib.debye_fit_init(ctypes.byref(h), ctypes.byref(o)) == D.DEBYE_EINVAL
    for cb, lanes in ((48, 0), (129, 0), (16, 1), (64, 4), (3, 8)):   # not whole warps, or > 128 threads
        o = D.default_options()
        o.cands_per_block, o.lanes_per_candidate = cb, lanes
        assert lib.debye_fit_init(ctypes.byref(h), ctypes.byref(o)) == D.DEBYE_EINVAL, (cb, lanes)
    for field, bad in (("de_cr", 1.5), ("de_f_lo", -0.1), ("de_f_hi", 0.25), ("de_strategy", 2),
                       ("da_t0", 0.0), ("da_qa", 1.0), ("solve_lanes", 2), ("solve_lanes", 16),
                       ("lanes_per_candidate", 3), ("lanes_per_candidate", 64)):
        o = D.default_options()
        setattr(o, field, bad)
        assert lib.debye_fit_init(ctypes.byref(h), ctypes.byref(o)) == D.DEBYE_EINVAL
    assert not h.value


def test_null_handle_calls(lib):
    assert lib.debye_fit_destroy(None) == D.DEBYE_OK
    assert lib.debye_eval_population(None, None, 1, 1, None, None, None, None, None) == D.DEBYE_EINVAL
    assert lib.debye_cost_grad(None, None, 1, 1, None, None, None, None, None) == D.DEBYE_EINVAL
    assert lib.debye_sync(None, None) == D.DEBYE_EINVAL
    assert lib.debye_version().startswith(b"debyefit")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "debyefit.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(debye_options), sizeof(debye_spectra), sizeof(debye_search));
  printf("%zu %zu %zu %zu\n", offsetof(debye_options, lam_search), offsetof(debye_options, lbfgs_c1),
         offsetof(debye_options, use_graphs), offsetof(debye_search, trace));
  printf("%zu\n", offsetof(debye_spectra, n_poles_host));
  printf("%zu %zu %zu\n", offsetof(debye_options, de_f_lo), offsetof(debye_options, de_strategy),
         offsetof(debye_search, method));
  printf("%zu %zu %zu\n", offsetof(debye_options, da_t0), offsetof(debye_options, da_qa),
         offsetof(debye_options, solve_lanes));
  printf("%zu\n", offsetof(debye_search, n_failed));
  return 0;
}
''')
    exe = tmp_path / "layout"
    cuda_inc = "/usr/local/cuda/include"
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cannot compile against cuda_runtime_api.h: " + r.stderr[:200])
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(D.Options)
    assert vals[1] == ctypes.sizeof(D.SpectraC)
    assert vals[2] == ctypes.sizeof(D.SearchC)
    assert vals[3] == D.Options.lam_search.offset
    assert vals[4] == D.Options.lbfgs_c1.offset
    assert vals[5] == D.Options.use_graphs.offset
    assert vals[6] == D.SearchC.trace.offset
    assert vals[7] == D.SpectraC.n_poles_host.offset
    assert vals[8] == D.Options.de_f_lo.offset
    assert vals[9] == D.Options.de_strategy.offset
    assert vals[10] == D.SearchC.method.offset
    assert vals[11] == D.Options.da_t0.offset and vals[12] == D.Options.da_qa.offset
    assert vals[13] == D.Options.solve_lanes.offset
    assert vals[14] == D.SearchC.n_failed.offset
