"""Batched multi-Debye fitting of dielectric spectra on GB300 (sm_103a).

The computation lives in the CUDA library libdebyefit.so (C ABI in
include/debyefit.h); `debyefit` is its thin ctypes binding.
"""
from .debyefit import (DebyeError, Handle, Spectra, cost_fn, debye_cost_grad, debye_eval_population,
                       debye_fit_batch, debye_sync, debye_synth_targets, lib, make_spectra)

__all__ = ["DebyeError", "Handle", "Spectra", "cost_fn", "debye_cost_grad", "debye_eval_population",
           "debye_fit_batch", "debye_sync", "debye_synth_targets", "lib", "make_spectra"]
