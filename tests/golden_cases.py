"""Reader of the hand-derived worked examples under tests/golden/ (Nside 1
and 2, lmax = mmax = 4): pixel centres, maps with their analysis
coefficients (Eq. 1) and coefficients with their synthesised maps (Eq. 2).
Expressions are evaluated with math's functions only; everything else in a
fixture is a comment."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NSIDES = (1, 2)
NSIDE, LMAX, MMAX = 1, 4, 4  # NSIDE: the default of the functions below
_NS = {"sqrt": math.sqrt, "pi": math.pi, "cos": math.cos, "sin": math.sin}


def _ev(expr, **var):
    return float(eval(expr, {"__builtins__": {}}, dict(_NS, **var)))


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln.split()


def pixels(nside=NSIDE):
    """[12 nside^2, 3]: z, sin(theta), phi of each pixel in RING order, from
    a per-pixel fixture or from the rings (pixels evenly spaced in phi from
    phi_0)."""
    if os.path.exists(os.path.join(GOLDEN, f"nside{nside}_pixels.txt")):
        rows = sorted((int(p), _ev(z), _ev(s), _ev(ph)) for p, z, s, ph in _lines(f"nside{nside}_pixels.txt"))
        assert [r[0] for r in rows] == list(range(12 * nside * nside))
        return np.array([r[1:] for r in rows])
    rings = sorted((int(i), _ev(z), _ev(s), int(n), _ev(p0)) for i, z, s, n, p0 in _lines(f"nside{nside}_rings.txt"))
    assert [r[0] for r in rings] == list(range(1, 4 * nside))
    px = [(z, s, p0 + 2 * math.pi * x / n) for _, z, s, n, p0 in rings for x in range(n)]
    assert len(px) == 12 * nside * nside
    return np.array(px)


def alm_index(l, m):
    """m-major packing: all l of m = 0, then of m = 1, ..."""
    return m * (2 * LMAX + 1 - m) // 2 + l


def nalm():
    return (MMAX + 1) * (LMAX + 1) - MMAX * (MMAX + 1) // 2


def _cases(name, nside):
    maps, alms, order = {}, {}, []
    for f in _lines(name):
        if f[0] == "map":
            maps[f[1]] = f[2]
            if f[1] not in order:
                order.append(f[1])
        elif f[0] == "alm":
            a = alms.setdefault(f[1], np.zeros(nalm(), np.complex128))
            a[alm_index(int(f[2]), int(f[3]))] = complex(_ev(f[4]), _ev(f[5]))
            if f[1] not in order:
                order.append(f[1])
        else:
            raise ValueError(f"unknown record {f[0]!r} in {name}")
    px = pixels(nside)
    out = []
    for k in order:
        m = np.array([_ev(maps[k], z=z, s=s, phi=ph) for z, s, ph in px])
        out.append((k, m, alms.get(k, np.zeros(nalm(), np.complex128))))
    return out


def analysis_cases(nside=NSIDE):
    """[(name, map [12 nside^2], alm [nalm])]: map in, coefficients out."""
    return _cases(f"nside{nside}_analysis.txt", nside)


def synthesis_cases(nside=NSIDE):
    """[(name, map [12 nside^2], alm [nalm])]: coefficients in, map out."""
    return _cases(f"nside{nside}_synthesis.txt", nside)
