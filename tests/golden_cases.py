"""Reader of the hand-derived worked examples under tests/golden/ (Nside 1,
lmax = mmax = 4): pixel centres, maps with their analysis coefficients
(Eq. 1) and coefficients with their synthesised maps (Eq. 2).  Expressions
are evaluated with math's functions only; everything else in a fixture is
a comment."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NSIDE, LMAX, MMAX = 1, 4, 4
_NS = {"sqrt": math.sqrt, "pi": math.pi, "cos": math.cos, "sin": math.sin}


def _ev(expr, **var):
    return float(eval(expr, {"__builtins__": {}}, dict(_NS, **var)))


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln.split()


def pixels():
    """[12, 3]: z, sin(theta), phi of each pixel in RING order."""
    rows = sorted((int(p), _ev(z), _ev(s), _ev(ph)) for p, z, s, ph in _lines("nside1_pixels.txt"))
    assert [r[0] for r in rows] == list(range(12 * NSIDE * NSIDE))
    return np.array([r[1:] for r in rows])


def alm_index(l, m):
    """m-major packing: all l of m = 0, then of m = 1, ..."""
    return m * (2 * LMAX + 1 - m) // 2 + l


def nalm():
    return (MMAX + 1) * (LMAX + 1) - MMAX * (MMAX + 1) // 2


def _cases(name):
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
    px = pixels()
    out = []
    for k in order:
        m = np.array([_ev(maps[k], z=z, s=s, phi=ph) for z, s, ph in px])
        out.append((k, m, alms.get(k, np.zeros(nalm(), np.complex128))))
    return out


def analysis_cases():
    """[(name, map [12], alm [nalm])]: map in, coefficients out."""
    return _cases("nside1_analysis.txt")


def synthesis_cases():
    """[(name, map [12], alm [nalm])]: coefficients in, map out."""
    return _cases("nside1_synthesis.txt")
