"""gprMax material commands in, multi-Debye material commands out (Sec. IV).

The paper's interface (Sec. IV, Listings 1 and 2): a dispersive material is
given by a command such as

    #havriliak_negami: f_lo f_hi alpha beta eps_inf d_eps tau0 sigma mu_r sigma_m N id [seed]

(frequency range in Hz, the relaxation function's parameters, then the basic
material properties: conductivity S/m, relative permeability, magnetic loss
Ohm/m; the number of Debye poles N, -1 for automatic; a text identifier; an
optional integer seed), and the fit is written back as

    #material: eps_inf sigma mu_r sigma_m id
    #add_dispersion_debye: N d_eps_1 tau_1 ... d_eps_N tau_N id

The paper names #jonscher, #crim and #raw_data without listing their
arguments; this module reads them as (same trailing fields as above):

    #jonscher: f_lo f_hi eps_inf a_p omega_p n_p sigma mu_r sigma_m N id [seed]
        eps_inf + a_p (w/omega_p)^(n_p-1) [1 - j cot(n_p pi/2)]
    #crim: f_lo f_hi a m f_1 .. f_m eps_inf_1 d_eps_1 tau_1 .. eps_inf_m d_eps_m tau_m
           sigma mu_r sigma_m N id [seed]
        (sum_i f_i eps_i^a)^(1/a) over m <= 3 Debye components (Eq. 6)
    #raw_data: file sigma mu_r sigma_m N id [seed]
        file: whitespace columns f (Hz), eps', eps'' (eps'' >= 0 for loss)

Targets of model commands are synthesised on the GPU (debye_synth_targets) at
K frequencies log-spaced over [f_lo, f_hi] (50 per decade, at least 50,
endpoints included); the relaxation times are searched in log10(tau) over
[floor(log10(1/(2 pi f_hi))) - 1, ceil(log10(1/(2 pi f_lo))) + 1]. All
commands with the same seed are fitted as one ragged batch (debye_fit_batch,
or debye_fit_auto for N = -1). Poles are written in ascending tau.
"""
from __future__ import annotations

import math
import os
import shlex
from dataclasses import dataclass, field

import numpy as np

from . import debyefit as D

MODEL_HN = 1
MODEL_JONSCHER = 4
MODEL_CRIM = 6
N_PARAMS = 16
POINTS_PER_DECADE = 50


@dataclass
class Command:
    kind: str                    # havriliak_negami | jonscher | crim | raw_data
    f_lo: float
    f_hi: float
    model: int                   # synthesis model id; -1 for raw data
    params: np.ndarray           # float64[N_PARAMS]
    sigma: str                   # basic material properties, echoed as given
    mu_r: str
    sigma_m: str
    n_poles: int                 # -1: automatic
    ident: str
    seed: int = 0
    data: np.ndarray | None = field(default=None, repr=False)   # raw data: (K, 3) f, eps', eps''


class CommandError(ValueError):
    pass


def _floats(tok, what):
    try:
        return [float(t) for t in tok]
    except ValueError as e:
        raise CommandError(f"{what}: {e}") from None


def _tail(tok, what):
    """sigma mu_r sigma_m N id [seed]"""
    if len(tok) not in (5, 6):
        raise CommandError(f"{what}: expected sigma mu_r sigma_m N id [seed], got {' '.join(tok)}")
    _floats(tok[:3], what)
    try:
        n = int(tok[3])
        seed = int(tok[5]) if len(tok) == 6 else 0
    except ValueError as e:
        raise CommandError(f"{what}: {e}") from None
    if n != -1 and not 1 <= n <= D.MAX_POLES:
        raise CommandError(f"{what}: number of poles {n} outside 1..{D.MAX_POLES} (or -1)")
    return tok[0], tok[1], tok[2], n, tok[4], seed


def parse_line(line: str, base_dir: str = ".") -> Command | None:
    """One command line (None for blank lines, comments and other commands)."""
    line = line.strip()
    if not line.startswith("#") or ":" not in line:
        return None
    name, _, rest = line[1:].partition(":")
    name = name.strip()
    tok = shlex.split(rest)
    p = np.zeros(N_PARAMS)
    if name == "havriliak_negami":
        if len(tok) < 12:
            raise CommandError(f"#havriliak_negami needs 12 or 13 arguments, got {len(tok)}")
        f_lo, f_hi, alpha, beta, eps_inf, d_eps, tau0 = _floats(tok[:7], name)
        if not (0.0 < alpha <= 1.0 and 0.0 < beta <= 1.0):
            raise CommandError(f"#havriliak_negami: alpha, beta must lie in (0, 1]")
        p[:5] = [eps_inf, d_eps, tau0, alpha, beta]
        return Command(name, f_lo, f_hi, MODEL_HN, p, *_tail(tok[7:], name))
    if name == "jonscher":
        if len(tok) < 11:
            raise CommandError(f"#jonscher needs 11 or 12 arguments, got {len(tok)}")
        f_lo, f_hi, eps_inf, a_p, omega_p, n_p = _floats(tok[:6], name)
        p[:4] = [eps_inf, a_p, omega_p, n_p]
        return Command(name, f_lo, f_hi, MODEL_JONSCHER, p, *_tail(tok[6:], name))
    if name == "crim":
        if len(tok) < 4:
            raise CommandError("#crim: too few arguments")
        f_lo, f_hi, a, m = _floats(tok[:4], name)
        m = int(m)
        if not 1 <= m <= 3:
            raise CommandError("#crim: 1 to 3 components")
        need = 4 + m + 3 * m
        if len(tok) < need + 5:
            raise CommandError(f"#crim with {m} components needs {need + 5} or {need + 6} arguments")
        vals = _floats(tok[4:need], name)
        p[0], p[1] = a, m
        p[2:2 + m] = vals[:m]
        for i in range(m):
            p[5 + 3 * i:8 + 3 * i] = vals[m + 3 * i:m + 3 * i + 3]
        return Command(name, f_lo, f_hi, MODEL_CRIM, p, *_tail(tok[need:], name))
    if name == "raw_data":
        if len(tok) < 6:
            raise CommandError("#raw_data needs file sigma mu_r sigma_m N id [seed]")
        path = tok[0] if os.path.isabs(tok[0]) else os.path.join(base_dir, tok[0])
        try:
            data = np.loadtxt(path, dtype=np.float64, ndmin=2)
        except OSError as e:
            raise CommandError(f"#raw_data: {e}") from None
        if data.shape[1] < 3 or data.shape[0] < 2:
            raise CommandError("#raw_data: the file needs rows of f eps' eps''")
        data = data[np.argsort(data[:, 0], kind="stable"), :3]
        if not np.all(data[:, 0] > 0):
            raise CommandError("#raw_data: frequencies must be positive")
        return Command(name, float(data[0, 0]), float(data[-1, 0]), -1, p, *_tail(tok[1:], name), data=data)
    return None


def parse(text: str, base_dir: str = ".") -> list[Command]:
    return [c for c in (parse_line(l, base_dir) for l in text.splitlines()) if c is not None]


def frequency_grid(f_lo: float, f_hi: float) -> np.ndarray:
    """Angular frequencies: POINTS_PER_DECADE per decade (at least 50), endpoints included."""
    if not (0.0 < f_lo < f_hi):
        raise CommandError("frequency range needs 0 < f_lo < f_hi")
    K = max(50, int(math.ceil(POINTS_PER_DECADE * math.log10(f_hi / f_lo))) + 1)
    return 2.0 * math.pi * np.logspace(math.log10(f_lo), math.log10(f_hi), K)


def tau_bounds(f_lo: float, f_hi: float) -> tuple[float, float]:
    lo = math.floor(math.log10(1.0 / (2.0 * math.pi * f_hi))) - 1.0
    hi = math.ceil(math.log10(1.0 / (2.0 * math.pi * f_lo))) + 1.0
    return lo, hi


def format_result(cmd: Command, eps_inf: float, d_eps, tau) -> str:
    """The #material and #add_dispersion_debye lines of one fit (Listing 2)."""
    pairs = " ".join(f"{d:.4f} {t:.4e}" for d, t in zip(d_eps, tau))
    return (f"#material: {eps_inf:.4f} {cmd.sigma} {cmd.mu_r} {cmd.sigma_m} {cmd.ident}\n"
            f"#add_dispersion_debye: {len(d_eps)} {pairs} {cmd.ident}")


def fit_commands(cmds: list[Command], precision: str = "mixed", P: int = 64, iters: int = 100,
                 polish_topk: int = 8, polish_iters: int = 50, method: str = "pso", device: str = "cuda"):
    """Fit every command; returns one dict per command: eps_inf, d_eps, tau (numpy), N,
    final_cost, and frac_err for automatic pole counts."""
    import torch
    results: list[dict | None] = [None] * len(cmds)
    for seed in sorted({c.seed for c in cmds}):
        idx = [i for i, c in enumerate(cmds) if c.seed == seed]
        for auto in (False, True):
            group = [i for i in idx if (cmds[i].n_poles == -1) == auto]
            if group:
                _fit_group([cmds[i] for i in group], group, results, auto, seed, precision, P, iters,
                           polish_topk, polish_iters, method, device)
    return results


def _fit_group(cmds, where, results, auto, seed, precision, P, iters, topk, polish_iters, method, device):
    import torch
    S = len(cmds)
    omegas = [frequency_grid(c.f_lo, c.f_hi) if c.model >= 0 else 2.0 * math.pi * c.data[:, 0] for c in cmds]
    offs = np.concatenate([[0], np.cumsum([o.size for o in omegas])]).astype(np.int64)
    omega = np.concatenate(omegas)
    npol = np.array([D.MAX_POLES if c.n_poles == -1 else c.n_poles for c in cmds], dtype=np.int32)
    bounds = np.array([tau_bounds(c.f_lo, c.f_hi) for c in cmds])
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
    om_d, offs_d = t(omega), t(offs, torch.int64)
    with D.Handle(precision) as h:
        # targets: model commands synthesised on the device, raw data copied in
        models = np.array([max(c.model, 0) for c in cmds], dtype=np.int32)
        params = np.stack([c.params for c in cmds])
        er, ei = D.debye_synth_targets(h, offs_d, om_d, t(models, torch.int32), t(params))
        raw = [i for i, c in enumerate(cmds) if c.model < 0]
        if raw:
            er_h, ei_h = er.cpu().numpy(), ei.cpu().numpy()
            for i in raw:
                er_h[offs[i]:offs[i + 1]] = cmds[i].data[:, 1]
                ei_h[offs[i]:offs[i + 1]] = cmds[i].data[:, 2]
            er, ei = t(er_h), t(ei_h)
        sp = D.Spectra(offs_d, om_d, er, ei, t(npol, torch.int32), t(bounds[:, 0]), t(bounds[:, 1]), offs, npol)
        n_max = int(npol.max())
        if auto:
            out = D.debye_fit_auto(h, sp, P=P, iters=iters, seed=seed, polish_topk=topk,
                                   polish_iters=polish_iters, n_max=n_max, method=method)
        else:
            out = D.debye_fit_batch(h, sp, P=P, iters=iters, seed=seed, polish_topk=topk,
                                    polish_iters=polish_iters, n_max=n_max, method=method)
        D.debye_sync(h)
    host = {k: v.cpu().numpy() for k, v in out.items()}
    for j, i in enumerate(where):
        N = int(host["n_chosen"][j]) if auto else int(npol[j])
        results[i] = {"eps_inf": float(host["eps_inf"][j]), "d_eps": host["d_eps"][j, :N].copy(),
                      "tau": host["tau"][j, :N].copy(), "N": N, "final_cost": float(host["final_cost"][j]),
                      "frac_err": float(host["frac_err"][j]) if auto else None}


def translate(text: str, base_dir: str = ".", **fit_kw) -> str:
    """Every material command of an input text replaced by its multi-Debye fit."""
    cmds = parse(text, base_dir)
    res = fit_commands(cmds, **fit_kw) if cmds else []
    return "\n".join(format_result(c, r["eps_inf"], r["d_eps"], r["tau"]) for c, r in zip(cmds, res))


def main(argv=None) -> int:
    import argparse
    ap = argparse.ArgumentParser(description="Fit gprMax dispersive-material commands with multi-Debye poles")
    ap.add_argument("input", help="text file with #havriliak_negami / #jonscher / #crim / #raw_data commands")
    ap.add_argument("--precision", default="mixed", choices=sorted(D.PRECISIONS))
    ap.add_argument("--method", default="pso", choices=["pso", "de", "da"])
    ap.add_argument("--population", type=int, default=64)
    ap.add_argument("--iters", type=int, default=100)
    args = ap.parse_args(argv)
    text = open(args.input).read()
    print(translate(text, os.path.dirname(os.path.abspath(args.input)), precision=args.precision,
                    method=args.method, P=args.population, iters=args.iters))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
