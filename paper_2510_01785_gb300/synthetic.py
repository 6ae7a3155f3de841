"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.

This module draws random numbers and lays them out; it holds none of the
transform's arithmetic.  The workloads follow the paper's use (Sec. IV-A:
fields band-limited to lmax = 3 Nside - 1; Sec. IV-C: a random complex
coefficient vector fitted to a target map):

* ``gaussian_alm``  -- Re and Im of a_lm ~ N(0, C_l) with C_l = (l+1)^-p,
                       a_l0 real, optional per-channel scale.
* ``white_maps``    -- i.i.d. N(0, 1) pixels.
* ``channel_scales``-- per-channel factors drawn uniformly from [lo, hi].
* ``poisson_arrivals`` -- arrival times of a Poisson request stream.

Coefficients are packed m-major: index m (2 lmax + 1 - m) / 2 + l, m >= 0.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2510017850


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def packed_l(lmax: int, mmax: int) -> np.ndarray:
    """l of every packed coefficient, in storage order."""
    return np.concatenate([np.arange(m, lmax + 1) for m in range(mmax + 1)])


def packed_m(lmax: int, mmax: int) -> np.ndarray:
    """m of every packed coefficient, in storage order."""
    return np.concatenate([np.full(lmax + 1 - m, m) for m in range(mmax + 1)])


def gaussian_alm(seed: int, lmax: int, mmax: int, nbatch: int, power: float = 2.0,
                 scales=None) -> np.ndarray:
    """complex128 [nbatch, nalm]; variance of Re and Im is (l+1)^-power;
    Im a_l0 = 0; each channel multiplied by scales[b] if given."""
    g = rng(seed)
    l = packed_l(lmax, mmax)
    m = packed_m(lmax, mmax)
    sd = (l + 1.0) ** (-0.5 * power)
    re = g.standard_normal((nbatch, l.size)) * sd
    im = g.standard_normal((nbatch, l.size)) * sd
    im[:, m == 0] = 0.0
    a = re + 1j * im
    if scales is not None:
        a *= np.asarray(scales, np.float64)[:, None]
    return a


def white_maps(seed: int, nside: int, nbatch: int) -> np.ndarray:
    """float64 [nbatch, 12 nside^2] of i.i.d. N(0, 1)."""
    return rng(seed).standard_normal((nbatch, 12 * nside * nside))


def channel_scales(seed: int, nbatch: int, lo: float = 1e-2, hi: float = 1e3) -> np.ndarray:
    return rng(seed).uniform(lo, hi, nbatch)


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    """Sorted arrival times (s) of a Poisson process of the given rate."""
    g = rng(seed)
    n = g.poisson(rate * duration)
    return np.sort(g.uniform(0.0, duration, n))
