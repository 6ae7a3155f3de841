"""FP64 CPU oracle for the HEALPix RING spherical harmonic transforms.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never imports, links or calls it, and the two share no code: this module wraps
``oracle.c`` (plain C, FP64, OpenMP) through ctypes.

Paper: arXiv 2510.01785 (cuHPX).  What each function follows:

* ``ring_geometry``          -- Sec. III-A grid structure (Gorski et al. pixel
                                centres, the grid's defining reference).
* ``lambda_chain``           -- Eq. 8 (orthonormal lambda_lm), Eq. 15
                                (Condon-Shortley phase), Eq. 16 (recurrence).
* ``ring_modes``             -- Eq. 13: per-ring Fourier sum at chosen m,
                                with the ring's phi_0 offset (Eq. 24/26).
* ``map2alm``                -- Eq. 26-27: a = Y^dagger W p, W = 4 pi / Npix
                                (Eq. 1 equal weights).
* ``alm2map``                -- Eq. 24-25: p = Y a.
* ``alm2map_adjoint``        -- Sec. III-F: adjoint of synthesis, Y^dagger.
* ``map2alm_adjoint``        -- Sec. III-F: adjoint of analysis, W Y.

Arrays: maps are float64 ``[nbatch, 12 nside^2]`` in RING order; coefficients
are complex128 ``[nbatch, nalm]`` with index ``m (2 lmax + 1 - m) / 2 + l``
(m >= 0 only, real fields).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# Test infrastructure: the planted-mistake tests run the pin suite in a
# subprocess against a modified build of oracle.c named by this variable.
_OVERRIDE = os.environ.get("HPX_ORACLE_LIB")
if _OVERRIDE:
    _LIB = _OVERRIDE
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it (gcc, OpenMP);
    with HPX_ORACLE_LIB set, use that library as it is."""
    if _OVERRIDE:
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int, ctypes.c_int64
            L.or_nalm.restype = i64
            L.or_nalm.argtypes = [i32, i32]
            L.or_max_threads.restype = i32
            L.or_ring_geometry.argtypes = [i32, P, P, P, P, P]
            L.or_lambda_chain.argtypes = [i32, i32, ctypes.c_double, ctypes.c_double, P]
            L.or_lambda_chain_log2.argtypes = [i32, i32, ctypes.c_double, ctypes.c_double, P, P]
            L.or_ring_modes.argtypes = [i32, i32, P, i32, P, P]
            L.or_map2alm_direct.argtypes = [i32, i32, i32, i32, P, P, P, i32]
            L.or_alm2map_direct.argtypes = [i32, i32, i32, i32, P, P, P, i32]
            L.or_map2alm_sep.argtypes = [i32, i32, i32, P, P, i32, P, P, P, i32]
            L.or_alm2map_sep.argtypes = [i32, i32, i32, i32, P, P, i32, P, P, i32]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def max_threads() -> int:
    return int(lib().or_max_threads())


# --------------------------------------------------------------------------
# indexing and geometry
# --------------------------------------------------------------------------
def nalm(lmax: int, mmax: int) -> int:
    return int(lib().or_nalm(lmax, mmax))


def alm_index(lmax: int, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def lm_arrays(lmax: int, mmax: int):
    """(l, m) of every packed coefficient, in storage order."""
    ls, ms = [], []
    for m in range(mmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls).astype(np.int32), np.concatenate(ms).astype(np.int32)


def ring_geometry(nside: int) -> dict:
    """Per ring (north to south): start pixel, pixel count, z = cos(theta),
    sin(theta) and the half-pixel shift sigma (phi_0 = sigma pi / N)."""
    R = 4 * nside - 1
    start = np.zeros(R, np.int64)
    nphi = np.zeros(R, np.int32)
    z = np.zeros(R, np.float64)
    sinth = np.zeros(R, np.float64)
    sigma = np.zeros(R, np.int32)
    lib().or_ring_geometry(nside, _ptr(start), _ptr(nphi), _ptr(z), _ptr(sinth), _ptr(sigma))
    return {"start": start, "nphi": nphi, "z": z, "sinth": sinth, "sigma": sigma}


def equal_weights(nside: int) -> np.ndarray:
    """Eq. 1: every pixel carries 4 pi / Npix."""
    return np.full(4 * nside - 1, 4.0 * np.pi / (12.0 * nside * nside))


def pixel_angles(nside: int):
    """theta, phi of every pixel centre in RING order (from ring_geometry)."""
    g = ring_geometry(nside)
    th, ph = [], []
    for y in range(4 * nside - 1):
        n = int(g["nphi"][y])
        x = np.arange(n)
        th.append(np.full(n, np.arctan2(g["sinth"][y], g["z"][y])))
        ph.append(np.pi * (2 * x + g["sigma"][y]) / n)
    return np.concatenate(th), np.concatenate(ph)


# --------------------------------------------------------------------------
# lambda_lm
# --------------------------------------------------------------------------
def lambda_chain(lmax: int, m: int, z: float, sinth: float) -> np.ndarray:
    """lambda_lm(z) for l = m..lmax (Eq. 8, 15, 16)."""
    out = np.zeros(lmax - m + 1, np.float64)
    lib().or_lambda_chain(lmax, m, float(z), float(sinth), _ptr(out))
    return out


def lambda_chain_log2(lmax: int, m: int, z: float, sinth: float):
    """log2|lambda_lm| and sign for l = m..lmax, without underflow."""
    lg = np.zeros(lmax - m + 1, np.float64)
    sg = np.zeros(lmax - m + 1, np.float64)
    lib().or_lambda_chain_log2(lmax, m, float(z), float(sinth), _ptr(lg), _ptr(sg))
    return lg, sg


def ring_modes(ring_values, sigma: int, ms) -> np.ndarray:
    """sum_x p_x exp(-i m phi_x), phi_x = pi (2x + sigma) / N, for each m."""
    p = np.ascontiguousarray(ring_values, np.float64)
    ms = np.ascontiguousarray(ms, np.int32)
    G = np.zeros(2 * len(ms), np.float64)
    lib().or_ring_modes(len(p), int(sigma), _ptr(p), len(ms), _ptr(ms), _ptr(G))
    return G[0::2] + 1j * G[1::2]


# --------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------
def _as_maps(maps):
    maps = np.ascontiguousarray(np.atleast_2d(maps), np.float64)
    return maps


def _as_alm(alm):
    alm = np.ascontiguousarray(np.atleast_2d(alm), np.complex128)
    return alm


def _weights(nside, w):
    if w is None:
        return None
    if isinstance(w, str):
        if w == "equal":
            return equal_weights(nside)
        raise ValueError(w)
    w = np.ascontiguousarray(w, np.float64)
    assert w.shape == (4 * nside - 1,)
    return w


def analysis_direct(maps, lmax, mmax, weights=None, nthreads=0):
    """Tier A: sum_y sum_x p_xy w_y lambda_lm exp(-i m phi_xy) for every
    coefficient (Eq. 26); weights=None means w = 1 (the operator Y^dagger)."""
    maps = _as_maps(maps)
    B, npix = maps.shape
    nside = int(round((npix / 12) ** 0.5))
    w = _weights(nside, weights)
    out = np.zeros((B, nalm(lmax, mmax)), np.complex128)
    lib().or_map2alm_direct(nside, lmax, mmax, B, _ptr(maps), _ptr(w),
                            _ptr(out.view(np.float64)), nthreads)
    return out


def synthesis_direct(alm, nside, lmax, mmax, scale=None, nthreads=0):
    """Tier A: Eq. 24 summed over +-m for every pixel, times scale[y]."""
    alm = _as_alm(alm)
    B = alm.shape[0]
    s = _weights(nside, scale)
    out = np.zeros((B, 12 * nside * nside), np.float64)
    lib().or_alm2map_direct(nside, lmax, mmax, B, _ptr(alm.view(np.float64)), _ptr(s),
                            _ptr(out), nthreads)
    return out


def analysis_sep(maps, lmax, ls, ms, weights=None, nthreads=0):
    """Tier B on chosen coefficients (l = ls[s], m = ms[s]); returns
    complex [nbatch, nsamp]."""
    maps = _as_maps(maps)
    B, npix = maps.shape
    nside = int(round((npix / 12) ** 0.5))
    w = _weights(nside, weights)
    ls = np.ascontiguousarray(ls, np.int32)
    ms = np.ascontiguousarray(ms, np.int32)
    assert ls.shape == ms.shape and np.all(ls >= ms) and np.all(ls <= lmax)
    out = np.zeros((B, len(ls)), np.complex128)
    lib().or_map2alm_sep(nside, lmax, B, _ptr(maps), _ptr(w), len(ls), _ptr(ls), _ptr(ms),
                         _ptr(out.view(np.float64)), nthreads)
    return out


def synthesis_sep(alm, nside, lmax, mmax, rings=None, scale=None, nthreads=0):
    """Tier B on chosen rings (all rings if None); returns [nbatch, sum N_y]
    with the rings' pixels back to back in the order given."""
    alm = _as_alm(alm)
    B = alm.shape[0]
    assert alm.shape[1] == nalm(lmax, mmax)
    R = 4 * nside - 1
    rings = np.arange(R, dtype=np.int32) if rings is None else np.ascontiguousarray(rings, np.int32)
    s = _weights(nside, scale)
    g = ring_geometry(nside)
    nout = int(np.sum(g["nphi"][rings]))
    out = np.zeros((B, nout), np.float64)
    lib().or_alm2map_sep(nside, lmax, mmax, B, _ptr(alm.view(np.float64)), _ptr(s),
                         len(rings), _ptr(rings), _ptr(out), nthreads)
    return out


def analysis(maps, lmax, mmax, weights=None, tier="sep", nthreads=0):
    if tier == "direct":
        return analysis_direct(maps, lmax, mmax, weights, nthreads)
    ls, ms = lm_arrays(lmax, mmax)
    return analysis_sep(maps, lmax, ls, ms, weights, nthreads)


def map2alm(maps, lmax, mmax, tier="sep", nthreads=0):
    """a = Y^dagger W p with equal weights 4 pi / Npix (Eq. 26-27, Eq. 1)."""
    return analysis(maps, lmax, mmax, "equal", tier, nthreads)


def alm2map(alm, nside, lmax, mmax, tier="sep", nthreads=0):
    """p = Y a (Eq. 24-25)."""
    if tier == "direct":
        return synthesis_direct(alm, nside, lmax, mmax, None, nthreads)
    return synthesis_sep(alm, nside, lmax, mmax, None, None, nthreads)


def map2alm_iter(maps, lmax, mmax, niter, nthreads=0):
    """Iterative refinement (Sec. II-A Eq. 4): a^0 = A f, then niter times
    r = f - S a^k and a^{k+1} = a^k + A r, with A = map2alm and S = alm2map.
    Returns the list [a^0, ..., a^niter]."""
    maps = _as_maps(maps)
    nside = int(round(np.sqrt(maps.shape[1] / 12)))
    a = map2alm(maps, lmax, mmax, nthreads=nthreads)
    out = [a]
    for _ in range(niter):
        r = maps - alm2map(a, nside, lmax, mmax, nthreads=nthreads)
        a = a + map2alm(r, lmax, mmax, nthreads=nthreads)
        out.append(a)
    return out


def alm2map_adjoint(maps, lmax, mmax, tier="sep", nthreads=0):
    """Y^dagger p: the adjoint of synthesis (Sec. III-F), i.e. the analysis
    sum with unit weights."""
    return analysis(maps, lmax, mmax, None, tier, nthreads)


def map2alm_adjoint(alm, nside, lmax, mmax, tier="sep", nthreads=0):
    """W Y a: the adjoint of analysis (Sec. III-F), synthesis scaled by the
    per-ring weight."""
    if tier == "direct":
        return synthesis_direct(alm, nside, lmax, mmax, "equal", nthreads)
    return synthesis_sep(alm, nside, lmax, mmax, None, "equal", nthreads)


def inner_full(a, b, lmax, mmax):
    """Real inner product over all +-m: sum_l Re(conj a_l0 b_l0)
    + 2 sum_{m>=1} Re(conj a_lm b_lm) (the product under which the
    adjoints of Sec. III-F are adjoint, for real fields)."""
    _, ms = lm_arrays(lmax, mmax)
    wt = np.where(ms == 0, 1.0, 2.0)
    return float(np.sum(wt * np.real(np.conj(a) * b)))


# ---------------------------------------------------------------------------
# pixel layouts (Sec. III-B), by geometry
# ---------------------------------------------------------------------------
_FACE_RING = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4])
_FACE_LON = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7])


def face_pixel_centres(nside):
    """(z, phi) of the centres of face pixels, array order [f][y][x] (the
    flat layout), from the inverse HEALPix projection (Gorski et al. 2005;
    Calabretta & Roukema 2007): the face is a square turned by 45 degrees in
    the (t, u) plane, centred at t = pi/4 * lon_f, u = pi/4 * (3 - ring_f),
    with x + y northward and x - y eastward; |u| <= pi/4 is the equatorial
    zone z = 8u / (3 pi), phi = t; beyond it sigma = 2 - 4|u|/pi,
    |z| = 1 - sigma^2/3 and phi = t_c + (t - t_c)/sigma about the face's
    central meridian t_c."""
    f, y, x = np.meshgrid(np.arange(12), np.arange(nside), np.arange(nside), indexing="ij")
    a, b = (x + 0.5) / nside, (y + 0.5) / nside
    tc = _FACE_LON[f] * np.pi / 4
    t = tc + np.pi / 4 * (a - b)
    u = (3 - _FACE_RING[f]) * np.pi / 4 + np.pi / 4 * (a + b - 1)
    z = 8 * u / (3 * np.pi)
    phi = t.copy()
    pol = np.abs(u) > np.pi / 4
    sig = 2 - 4 * np.abs(u[pol]) / np.pi
    z[pol] = np.sign(u[pol]) * (1 - sig ** 2 / 3)
    phi[pol] = tc[pol] + (t[pol] - tc[pol]) / sig
    return z.ravel(), np.mod(phi.ravel(), 2 * np.pi)


def _morton(x, y):
    """Interleave: x to the even bits, y to the odd bits."""
    out = np.zeros_like(x)
    for bit in range(16):
        out |= ((x >> bit) & 1) << (2 * bit)
        out |= ((y >> bit) & 1) << (2 * bit + 1)
    return out


def layout_permutations(nside):
    """For every flat-order pixel [f][y][x]: its RING index (by matching its
    geometric centre to the ring pixel centres of Sec. III-A), its NESTED
    index (f nside^2 + Morton(x, y)) and its FLAT index."""
    z, phi = face_pixel_centres(nside)
    g = ring_geometry(nside)
    zr = np.asarray(g["z"])
    ring = np.argmin(np.abs(z[:, None] - zr[None, :]), axis=1)
    N, sig = np.asarray(g["nphi"])[ring], np.asarray(g["sigma"])[ring]
    k = np.mod(np.rint((phi * N / np.pi - sig) / 2).astype(np.int64), N)
    ring_idx = np.asarray(g["start"])[ring] + k
    f, y, x = np.meshgrid(np.arange(12), np.arange(nside), np.arange(nside), indexing="ij")
    nest_idx = (f * nside * nside + _morton(x, y)).ravel()
    flat_idx = np.arange(12 * nside * nside)
    return {"ring": ring_idx.astype(np.int64), "nested": nest_idx.astype(np.int64), "flat": flat_idx}


def layout_index(nside, src, dst):
    """index[t] = the src index of the pixel whose dst index is t."""
    perm = layout_permutations(nside)
    idx = np.empty(12 * nside * nside, np.int64)
    idx[perm[dst]] = perm[src]
    return idx
