"""Counter-based random numbers for the seeded search (oracle).

The paper only says that each command takes an optional integer seed for the
stochastic optimiser (Sec. IV). Reading: every random number is a pure
function of (seed, stream tag, spectrum, generation, particle, dimension),
so that a population does not depend on evaluation order or batching.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a mixing function:
    z += 0x9E3779B97F4A7C15
    z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z  =  z ^ (z >> 31)
all modulo 2^64. The key is absorbed one field at a time,
    h = mix(seed); h = mix(h ^ tag); h = mix(h ^ spectrum);
    h = mix(h ^ generation); h = mix(h ^ particle); h = mix(h ^ dim),
and the uniform double is (h >> 11) * 2^-53 in [0, 1). An integer below m
(m < 2^32) is ((h >> 32) * m) >> 32, the multiply-shift map of the key's upper
32 bits (Lemire, "Fast random integer generation in an interval", 2019,
without the rejection step; the bias is below m / 2^32).
"""
from __future__ import annotations

MASK = (1 << 64) - 1

TAG_INIT_POS = 1
TAG_INIT_VEL = 2
TAG_R1 = 3
TAG_R2 = 4
TAG_DE_IDX = 5     # differential evolution: donor indices
TAG_DE_J = 6       # the coordinate always taken from the mutant
TAG_DE_CR = 7      # binomial crossover draws
TAG_DE_BOUND = 8   # re-draw of a mutant coordinate outside the bounds
TAG_DE_F = 9       # per-generation scale factor (dither)
TAG_DA_VISIT = 10  # dual annealing: uniforms of the visiting deviates
TAG_DA_ACCEPT = 11 # dual annealing: acceptance draws


def mix(z: int) -> int:
    """One SplitMix64 step applied to z (mod 2^64)."""
    z = (z + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def key(seed: int, tag: int, spectrum: int, generation: int, particle: int, dim: int) -> int:
    h = mix(seed & MASK)
    h = mix(h ^ tag)
    h = mix(h ^ spectrum)
    h = mix(h ^ generation)
    h = mix(h ^ particle)
    return mix(h ^ dim)


def uniform(seed: int, tag: int, spectrum: int, generation: int, particle: int, dim: int) -> float:
    """Uniform double in [0, 1) for the given counter."""
    return (key(seed, tag, spectrum, generation, particle, dim) >> 11) * (1.0 / (1 << 53))


def below(z: int, m: int) -> int:
    """Integer in [0, m) from the key z (multiply-shift of the upper 32 bits)."""
    return ((z >> 32) * m) >> 32


def mix_array(z):
    """`mix` over a numpy uint64 array (wrap-around arithmetic mod 2^64)."""
    import numpy as np
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def key_array(seed: int, tag: int, spectrum: int, generation: int, P: int, N: int):
    """key(seed, tag, spectrum, generation, p, d) for all p < P, d < N, as uint64 (P, N)."""
    import numpy as np
    h = mix(seed & MASK)
    h = mix(h ^ tag)
    h = mix(h ^ (spectrum & MASK))
    h = mix(h ^ (generation & MASK))
    hp = mix_array(np.uint64(h) ^ np.arange(P, dtype=np.uint64))
    return mix_array(hp[:, None] ^ np.arange(N, dtype=np.uint64)[None, :])


def uniform_cols(seed: int, tag: int, spectrum: int, generation: int, P: int, cols):
    """uniform(seed, tag, spectrum, generation, p, c) for all p < P and c in cols, as (P, len(cols))."""
    import numpy as np
    h = mix(seed & MASK)
    h = mix(h ^ tag)
    h = mix(h ^ (spectrum & MASK))
    h = mix(h ^ (generation & MASK))
    hp = mix_array(np.uint64(h) ^ np.arange(P, dtype=np.uint64))
    hd = mix_array(hp[:, None] ^ np.asarray(cols, dtype=np.uint64)[None, :])
    return (hd >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_array(seed: int, tag: int, spectrum: int, generation: int, P: int, N: int):
    """uniform(seed, tag, spectrum, generation, p, d) for all p < P, d < N, as (P, N)."""
    import numpy as np
    hd = key_array(seed, tag, spectrum, generation, P, N)
    return (hd >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
