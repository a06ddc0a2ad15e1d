"""Elementary functions with a fixed sequence of IEEE double operations (oracle).

Dual annealing (Sec. III-B) draws its moves from a heavy-tailed visiting
distribution and accepts uphill moves with a generalized Metropolis rule; both
need log and exp, and a Gaussian deviate. Library exp/log differ between
implementations in the last bits, and a different last bit can flip an
acceptance decision. These functions are instead defined by an explicit
sequence of correctly rounded double operations (+, -, *, /, sqrt, and exact
frexp/ldexp/rint/fmod), so that any implementation performing the same
sequence, without fused multiply-add, returns the same bits. Accuracy is a few
ulp (tests pin them against math.log / math.exp).

    log(x), x > 0:  x = m 2^e with m in [sqrt(1/2), sqrt(2)); f = (m-1)/(m+1);
                    log x = e ln2 + 2 f sum_{j=0}^{12} f^(2j) / (2j+1)
                    (the atanh series, Horner in f^2 from j = 12 down).
    exp(x):         k = rint(x / ln2), r = (x - k ln2_hi) - k ln2_lo (|r| <= ln2/2;
                    ln2_hi has 32 significant bits, so k ln2_hi is exact);
                    exp x = 2^k (1 + r (1 + r/2 (1 + r/3 (... (1 + r/14)))))
                    (Taylor, Horner from the degree-14 term).
    Gaussian pair:  Marsaglia's polar method on u, v = 2U - 1 with
                    s = u^2 + v^2 in (0, 1): (u, v) sqrt(-2 log s / s).
Every function works elementwise on numpy arrays (numpy's float64 array
arithmetic is IEEE, without fusion) and on Python floats.
"""
from __future__ import annotations

import numpy as np

LN2 = 0.6931471805599453          # ln 2 rounded to double
LN2_HI = 0.6931471803691238       # ln 2 with the low 21 mantissa bits cleared (0x1.62e42feep-1)
LN2_LO = 1.9082149292705877e-10   # ln 2 - LN2_HI, rounded to double (from 50-digit ln 2)
SQRT_HALF = 0.7071067811865476    # sqrt(1/2) rounded to double
LOG_TERMS = 13                    # j = 0..12
EXP_TERMS = 14                    # degree of the Taylor polynomial
EXP_MAX = 709.0                   # larger arguments overflow: +inf
EXP_MIN = -745.0                  # smaller arguments underflow: 0


def log(x):
    """Natural logarithm for x > 0 (finite); elementwise."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, m in [0.5, 1)
    low = m < SQRT_HALF
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    f = (m - 1.0) / (m + 1.0)
    s = f * f
    p = np.full_like(f, 1.0 / (2 * (LOG_TERMS - 1) + 1))
    for j in range(LOG_TERMS - 2, -1, -1):
        p = p * s + 1.0 / (2 * j + 1)
    out = e * LN2 + (2.0 * f) * p
    return out if out.ndim else float(out)


def exp(x):
    """Exponential; +inf above EXP_MAX, 0 below EXP_MIN; elementwise."""
    x = np.asarray(x, dtype=np.float64)
    xc = np.clip(x, EXP_MIN, EXP_MAX)
    k = np.rint(xc / LN2)
    r = (xc - k * LN2_HI) - k * LN2_LO
    p = np.ones_like(r)
    for j in range(EXP_TERMS, 0, -1):
        p = 1.0 + (p * r) / float(j)
    out = np.ldexp(p, k.astype(np.int64))
    out = np.where(x > EXP_MAX, np.inf, np.where(x < EXP_MIN, 0.0, out))
    return out if out.ndim else float(out)


POLAR_TRIES = 32


def gauss_pair(u_list, v_list):
    """Standard normal pair by the polar method from uniform draws in [0, 1):
    u_list[t], v_list[t] are the draws of try t (arrays of equal shape); the first
    try with 0 < s < 1 is used. Returns (z1, z2); (0, 0) where every try failed."""
    z1 = None
    done = None
    for t in range(len(u_list)):
        u = 2.0 * np.asarray(u_list[t], dtype=np.float64) - 1.0
        v = 2.0 * np.asarray(v_list[t], dtype=np.float64) - 1.0
        s = u * u + v * v
        ok = (s > 0.0) & (s < 1.0)
        sl = np.where(ok, s, 0.5)
        f = np.sqrt((-2.0 * log(sl)) / sl)
        if z1 is None:
            z1 = np.zeros_like(u)
            z2 = np.zeros_like(u)
            done = np.zeros(u.shape, dtype=bool)
        take = ok & ~done
        z1 = np.where(take, u * f, z1)
        z2 = np.where(take, v * f, z2)
        done = done | ok
    return z1, z2
