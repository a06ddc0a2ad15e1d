"""Python binding of libdebyefit (ctypes): argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors
into the plain pointers and sizes of the C ABI (include/debyefit.h) and back.
PyTorch provides device memory and streams. There is no CPU fallback: if the
library is not built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdebyefit.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "debyefit.h")

DEBYE_OK = 0
DEBYE_EINVAL = -1
DEBYE_ECUDA = -2
DEBYE_ENOMEM = -3
DEBYE_ETIMEOUT = -4
DEBYE_EINTERNAL = -5
DEBYE_ENOTFINITE = -6
DEBYE_EBOUNDS = -7
PREC_FP64 = 0
PREC_MIXED = 1
PREC_FP64_SUMS = 2
PREC_MIXED_TABLE = 3
PRECISIONS = {"mixed": PREC_MIXED, "fp64": PREC_FP64, "fp64_sums": PREC_FP64_SUMS,
              "mixed_table": PREC_MIXED_TABLE}
SEARCH_PSO = 0
SEARCH_DE = 1
SEARCH_DA = 2
DE_RAND1 = 0
DE_BEST1 = 1
MAX_POLES = 20
N_PARAMS = 16


class DebyeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"debyefit error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("lam_search", ctypes.c_double), ("lam_final", ctypes.c_double),
                ("pso_omega", ctypes.c_double), ("pso_phi_p", ctypes.c_double),
                ("pso_phi_g", ctypes.c_double), ("lbfgs_m", ctypes.c_int32),
                ("lbfgs_max_trials", ctypes.c_int32), ("lbfgs_c1", ctypes.c_double),
                ("cands_per_block", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("de_f_lo", ctypes.c_double), ("de_f_hi", ctypes.c_double), ("de_cr", ctypes.c_double),
                ("de_strategy", ctypes.c_int32), ("da_t0", ctypes.c_double), ("da_qa", ctypes.c_double),
                ("solve_lanes", ctypes.c_int32), ("lanes_per_candidate", ctypes.c_int32)]


class SpectraC(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int64), ("offsets", ctypes.c_void_p), ("omega", ctypes.c_void_p),
                ("eps_re", ctypes.c_void_p), ("eps_im", ctypes.c_void_p),
                ("n_poles", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("offsets_host", ctypes.c_void_p), ("n_poles_host", ctypes.c_void_p)]


class SearchC(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("iters", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("polish_topk", ctypes.c_int32), ("polish_iters", ctypes.c_int32),
                ("trace", ctypes.c_void_p), ("evals", ctypes.c_void_p), ("method", ctypes.c_int32),
                ("n_failed", ctypes.c_void_p)]


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int


def lib() -> ctypes.CDLL:
    """Load libdebyefit.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.debye_default_options.argtypes = [ctypes.POINTER(Options)]
    L.debye_default_options.restype = None
    L.debye_fit_init.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Options)]
    L.debye_fit_destroy.argtypes = [_VP]
    L.debye_synth_targets.argtypes = [_VP, ctypes.c_int64] + [_VP] * 11 + [_VP]
    L.debye_eval_population.argtypes = [_VP, ctypes.POINTER(SpectraC), ctypes.c_int32, ctypes.c_int32,
                                        _VP, _VP, _VP, _VP, _VP]
    L.debye_cost_grad.argtypes = [_VP, ctypes.POINTER(SpectraC), ctypes.c_int32, ctypes.c_int32,
                                  _VP, _VP, _VP, _VP, _VP]
    L.debye_fit_batch.argtypes = [_VP, ctypes.POINTER(SpectraC), ctypes.POINTER(SearchC), ctypes.c_int32,
                                  _VP, _VP, _VP, _VP, _VP]
    L.debye_fit_auto.argtypes = [_VP, ctypes.POINTER(SpectraC), ctypes.POINTER(SearchC), ctypes.c_int32,
                                 ctypes.c_double, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP]
    L.debye_sync.argtypes = [_VP, _VP]
    L.debye_check_bounded_wait.argtypes = [_VP, _VP]
    L.debye_last_error.argtypes = [_VP]
    L.debye_last_error.restype = ctypes.c_char_p
    L.debye_version.restype = ctypes.c_char_p
    L.debye_profile_enable.argtypes = [_VP, ctypes.c_int32]
    L.debye_launch_count.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
    L.debye_autotune.argtypes = [_VP, ctypes.POINTER(SpectraC), ctypes.c_int32, ctypes.c_int32, _VP, _VP,
                                 ctypes.c_char_p, _VP, _VP]
    L.debye_eval_population_noalloc.argtypes = [ctypes.POINTER(Options), ctypes.POINTER(SpectraC),
                                                ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP,
                                                ctypes.c_char_p, ctypes.c_int32, _VP]
    L.debye_profile_read.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    for f in ("debye_fit_init", "debye_fit_destroy", "debye_synth_targets", "debye_eval_population",
              "debye_cost_grad", "debye_fit_batch", "debye_sync", "debye_profile_enable",
              "debye_profile_read", "debye_launch_count", "debye_autotune", "debye_eval_population_noalloc",
              "debye_check_bounded_wait"):
        getattr(L, f).restype = _I
    _lib = L
    return L


def header_functions() -> list[str]:
    """Names of the functions declared in include/debyefit.h."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(debye_\w+)\s*\(", txt, re.M)))


def _check_n_max(theta, n_max):
    """The kernels stride theta [S, P, n_max] rows by n_max: it must be theta's last extent."""
    nm = theta.shape[2]
    if n_max is not None and n_max != nm:
        raise ValueError(f"n_max = {n_max} differs from theta.shape[2] = {nm}")
    return nm


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def default_options() -> Options:
    o = Options()
    lib().debye_default_options(ctypes.byref(o))
    return o


class Handle:
    """debye_handle with its options (precision 'mixed', 'fp64', 'fp64_sums' or 'mixed_table')."""

    def __init__(self, precision: str = "mixed", **opts):
        o = default_options()
        o.precision = PRECISIONS[precision]
        for k, v in opts.items():
            setattr(o, k, v)
        self.options = o
        self._h = _VP()
        rc = lib().debye_fit_init(ctypes.byref(self._h), ctypes.byref(o))
        if rc != DEBYE_OK:
            raise DebyeError(rc, "debye_fit_init failed")

    @property
    def ptr(self):
        return self._h

    def check(self, rc: int):
        if rc != DEBYE_OK:
            raise DebyeError(rc, lib().debye_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().debye_fit_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


@dataclass
class Spectra:
    """A ragged batch on the device (torch tensors) plus host copies of offsets and N."""
    offsets: object
    omega: object
    eps_re: object
    eps_im: object
    n_poles: object
    lo: object
    hi: object
    offsets_host: np.ndarray
    n_poles_host: np.ndarray

    @property
    def S(self) -> int:
        return int(self.n_poles_host.shape[0])

    @property
    def n_max(self) -> int:
        return int(self.n_poles_host.max()) if self.S else 1

    def c(self) -> SpectraC:
        return SpectraC(self.S, _ptr(self.offsets), _ptr(self.omega), _ptr(self.eps_re),
                        _ptr(self.eps_im), _ptr(self.n_poles), _ptr(self.lo), _ptr(self.hi),
                        self.offsets_host.ctypes.data, self.n_poles_host.ctypes.data)


def make_spectra(offsets, omega, eps_re, eps_im, n_poles, lo, hi, device="cuda") -> Spectra:
    """Spectra from host arrays (copied to `device`)."""
    import torch
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    npol = np.ascontiguousarray(n_poles, dtype=np.int32)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
    return Spectra(t(offs, torch.int64), t(omega, torch.float64), t(eps_re, torch.float64),
                   t(eps_im, torch.float64), t(npol, torch.int32), t(lo, torch.float64),
                   t(hi, torch.float64), offs, npol)


# ------------------------------------------------------------------ entry points (C ABI names)

def debye_synth_targets(h: Handle, offsets, omega, model, params, pole_offsets=None, pole_tau=None,
                        pole_deps=None, noise_re=None, noise_im=None, stream=None):
    """eps', eps'' (device tensors) of every spectrum from model ids and parameter records."""
    import torch
    n = omega.shape[0]
    er = torch.empty(n, dtype=torch.float64, device=omega.device)
    ei = torch.empty(n, dtype=torch.float64, device=omega.device)
    S = model.shape[0]
    h.check(lib().debye_synth_targets(h.ptr, S, _ptr(offsets), _ptr(omega), _ptr(model), _ptr(params),
                                      _ptr(pole_offsets), _ptr(pole_tau), _ptr(pole_deps), _ptr(noise_re),
                                      _ptr(noise_im), _ptr(er), _ptr(ei), _stream(stream)))
    return er, ei


def debye_eval_population(h: Handle, sp: Spectra, theta, weights: bool = False, n_max: int | None = None,
                          cost=None, weights_out=None, n_failed=None, stream=None):
    """Cost [S, P] (and weights [S, P, n_max+1]) of the population theta [S, P, n_max].
    n_failed: optional int32 [S] device tensor, incremented per candidate whose damped
    matrix is not positive definite."""
    import torch
    S, P, nm = theta.shape
    n_max = _check_n_max(theta, n_max)
    assert theta.dtype == torch.float64 and theta.is_contiguous()
    if cost is None:
        cost = torch.empty((S, P), dtype=torch.float64, device=theta.device)
    if weights and weights_out is None:
        weights_out = torch.empty((S, P, n_max + 1), dtype=torch.float64, device=theta.device)
    c = sp.c()
    h.check(lib().debye_eval_population(h.ptr, ctypes.byref(c), P, n_max, _ptr(theta), _ptr(cost),
                                        _ptr(weights_out) if weights else None, _ptr(n_failed), _stream(stream)))
    return (cost, weights_out) if weights else cost


def debye_cost_grad(h: Handle, sp: Spectra, theta, cost=None, grad=None, n_failed=None, stream=None):
    """Cost [S, P] and d cost / d theta [S, P, n_max] (n_failed as for debye_eval_population)."""
    import torch
    S, P, nm = theta.shape
    if cost is None:
        cost = torch.empty((S, P), dtype=torch.float64, device=theta.device)
    if grad is None:
        grad = torch.empty_like(theta)
    c = sp.c()
    h.check(lib().debye_cost_grad(h.ptr, ctypes.byref(c), P, nm, _ptr(theta), _ptr(cost), _ptr(grad),
                                  _ptr(n_failed), _stream(stream)))
    return cost, grad


def debye_fit_batch(h: Handle, sp: Spectra, P: int, iters: int, seed: int = 0, polish_topk: int = 8,
                    polish_iters: int = 50, n_max: int | None = None, trace: bool = False, stream=None,
                    out=None, method: str = "pso", n_failed: bool = False):
    """Whole fit of every spectrum: dict of eps_inf [S], d_eps [S, n_max], tau [S, n_max],
    final_cost [S], evals (candidate evaluations x K), optionally trace [S, iters+1] and
    n_failed [S] (int32: candidates whose damped matrix was not positive definite).
    method: "pso" (particle swarm), "de" (differential evolution) or "da" (dual annealing)."""
    import torch
    dev = sp.omega.device
    n_max = sp.n_max if n_max is None else n_max
    S = sp.S
    if out is None:
        out = {"eps_inf": torch.empty(S, dtype=torch.float64, device=dev),
               "d_eps": torch.empty((S, n_max), dtype=torch.float64, device=dev),
               "tau": torch.empty((S, n_max), dtype=torch.float64, device=dev),
               "final_cost": torch.empty(S, dtype=torch.float64, device=dev),
               "evals": torch.zeros(1, dtype=torch.float64, device=dev)}
        if trace:
            out["trace"] = torch.empty((S, iters + 1), dtype=torch.float64, device=dev)
        if n_failed:
            out["n_failed"] = torch.zeros(S, dtype=torch.int32, device=dev)
    elif "n_failed" in out:
        out["n_failed"].zero_()
    srch = SearchC(P, iters, seed, polish_topk, polish_iters, _ptr(out.get("trace")), _ptr(out["evals"]),
                   {"pso": SEARCH_PSO, "de": SEARCH_DE, "da": SEARCH_DA}[method], _ptr(out.get("n_failed")))
    c = sp.c()
    h.check(lib().debye_fit_batch(h.ptr, ctypes.byref(c), ctypes.byref(srch), n_max, _ptr(out["eps_inf"]),
                                  _ptr(out["d_eps"]), _ptr(out["tau"]), _ptr(out["final_cost"]),
                                  _stream(stream)))
    return out


def debye_fit_auto(h: Handle, sp: Spectra, P: int, iters: int, seed: int = 0, polish_topk: int = 8,
                   polish_iters: int = 50, n_max: int | None = None, threshold: float = 5.0, wave: int = 4,
                   method: str = "pso", stream=None):
    """Automatic pole count: sp.n_poles is each spectrum's cap; returns the dict of
    debye_fit_batch plus frac_err [S] (percent) and n_chosen [S] (int32)."""
    import torch
    dev = sp.omega.device
    n_max = sp.n_max if n_max is None else n_max
    S = sp.S
    f64 = dict(dtype=torch.float64, device=dev)
    out = {"eps_inf": torch.empty(S, **f64), "d_eps": torch.empty((S, n_max), **f64),
           "tau": torch.empty((S, n_max), **f64), "final_cost": torch.empty(S, **f64),
           "frac_err": torch.empty(S, **f64), "n_chosen": torch.empty(S, dtype=torch.int32, device=dev),
           "evals": torch.zeros(1, **f64)}
    srch = SearchC(P, iters, seed, polish_topk, polish_iters, None, _ptr(out["evals"]),
                   {"pso": SEARCH_PSO, "de": SEARCH_DE, "da": SEARCH_DA}[method], None)
    c = sp.c()
    h.check(lib().debye_fit_auto(h.ptr, ctypes.byref(c), ctypes.byref(srch), n_max, float(threshold), wave,
                                 _ptr(out["eps_inf"]), _ptr(out["d_eps"]), _ptr(out["tau"]),
                                 _ptr(out["final_cost"]), _ptr(out["frac_err"]), _ptr(out["n_chosen"]),
                                 _stream(stream)))
    return out


def debye_sync(h: Handle, stream=None):
    h.check(lib().debye_sync(h.ptr, _stream(stream)))


def debye_check_bounded_wait(h: Handle, stream=None):
    """Enqueue the failure-path check of the bounded device waits: the next debye_sync
    raises DebyeError with code DEBYE_ETIMEOUT (after about 1 s)."""
    h.check(lib().debye_check_bounded_wait(h.ptr, _stream(stream)))


KERNEL_KINDS = {"gram": 0, "refine": 1, "grad": 2, "solve": 3, "finish": 4, "gram_masked": 5,
                "refine_masked": 6, "grad_masked": 7, "sums": 8, "sums_masked": 9, "table": 10,
                "table_eval": 11}


def debye_eval_population_noalloc(sp: Spectra, theta, precision: str = "mixed", weights: bool = False,
                                  n_max: int | None = None, options: Options | None = None, cost=None,
                                  weights_out=None, stream=None):
    """debye_eval_population without a handle and without any device allocation by the
    library (fixed scratch inside the library); the caller provides the outputs."""
    import torch
    S, P, nm = theta.shape
    n_max = _check_n_max(theta, n_max)
    o = options if options is not None else default_options()
    o.precision = PRECISIONS[precision]
    if cost is None:
        cost = torch.empty((S, P), dtype=torch.float64, device=theta.device)
    if weights and weights_out is None:
        weights_out = torch.empty((S, P, n_max + 1), dtype=torch.float64, device=theta.device)
    buf = ctypes.create_string_buffer(512)
    c = sp.c()
    rc = lib().debye_eval_population_noalloc(ctypes.byref(o), ctypes.byref(c), P, n_max, _ptr(theta),
                                             _ptr(cost), _ptr(weights_out) if weights else None, buf, 512,
                                             _stream(stream))
    if rc != DEBYE_OK:
        raise DebyeError(rc, buf.value.decode())
    return (cost, weights_out) if weights else cost


def debye_autotune(h: Handle, sp: Spectra, theta, cache_path: str | None = None, stream=None) -> dict:
    """Time the work layouts on this batch and keep the fastest for h: returns
    {"cands_per_block", "lanes_per_candidate"} of full populations and
    {"polish_cands_per_block", "polish_lanes_per_candidate"} of the polish's accepted points."""
    import torch
    S, P, nm = theta.shape
    cost = torch.empty((S, P), dtype=torch.float64, device=theta.device)
    chosen = (ctypes.c_int32 * 4)()
    c = sp.c()
    h.check(lib().debye_autotune(h.ptr, ctypes.byref(c), P, nm, _ptr(theta), _ptr(cost),
                                 cache_path.encode() if cache_path else None, chosen, _stream(stream)))
    return {"cands_per_block": chosen[0], "lanes_per_candidate": chosen[1],
            "polish_cands_per_block": chosen[2], "polish_lanes_per_candidate": chosen[3]}


def debye_launch_count(h: Handle, reset: bool = False) -> int:
    """Kernel launches enqueued by the handle so far."""
    n = ctypes.c_int64()
    h.check(lib().debye_launch_count(h.ptr, ctypes.byref(n), 1 if reset else 0))
    return n.value


def debye_profile_enable(h: Handle, enable: bool = True):
    h.check(lib().debye_profile_enable(h.ptr, 1 if enable else 0))


def debye_profile_read(h: Handle) -> dict:
    """{kind: (launches, ms, flops)} accumulated since timing was enabled."""
    out = {}
    for name, k in KERNEL_KINDS.items():
        n, ms, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        h.check(lib().debye_profile_read(h.ptr, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl)))
        out[name] = (n.value, ms.value, fl.value)
    return out


def version() -> str:
    return lib().debye_version().decode()


# ------------------------------------------------------------------ autograd

def _autograd_fn():
    import torch

    class CostGrad(torch.autograd.Function):
        """cost(theta) with the VarPro gradient computed by the library (debye_cost_grad)."""

        @staticmethod
        def forward(ctx, theta, h, sp):
            cost, grad = debye_cost_grad(h, sp, theta.detach().contiguous())
            ctx.save_for_backward(grad)
            return cost

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout[..., None] * grad, None, None

    return CostGrad


def cost_fn(theta, h: Handle, sp: Spectra):
    """Differentiable DLS cost of theta [S, P, n_max] (torch.autograd)."""
    return _autograd_fn().apply(theta, h, sp)
