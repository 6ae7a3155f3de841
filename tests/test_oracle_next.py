"""Pins of the oracle's functions for the next rows of the path: iterative
refinement (Sec. II-A Eq. 4)."""
import numpy as np

import oracle
from paper_2510_01785_gb300 import synthetic as syn


def _norms(x):
    return np.linalg.norm(np.atleast_2d(x), axis=1)


def test_refinement_residual_decreases_and_converges():
    """For a band-limited map f = S a_true (lmax below the grid's exact range),
    every refinement step lowers ||f - S a^k|| and ||a^k - a_true||."""
    nside, lmax = 8, 15
    a_true = syn.gaussian_alm(501, lmax, lmax, 2, power=1.0)
    f = oracle.alm2map(a_true, nside, lmax, lmax)
    its = oracle.map2alm_iter(f, lmax, lmax, 4)
    res = [_norms(f - oracle.alm2map(a, nside, lmax, lmax)) for a in its]
    err = [_norms(a - a_true) for a in its]
    for k in range(4):
        assert np.all(res[k + 1] < res[k]), (k, res[k], res[k + 1])
        assert np.all(err[k + 1] < err[k]), (k, err[k], err[k + 1])
    # equal-weight quadrature leaves a visible first-step error that refinement removes
    assert np.all(err[0] > 1e-4 * _norms(a_true)) and np.all(err[4] < 0.1 * err[0])


def test_refinement_residual_decreases_at_full_band():
    """At lmax = 3 nside - 1 (not exactly solvable) the residual still falls."""
    nside, lmax = 8, 23
    f = syn.white_maps(502, nside, 2)
    its = oracle.map2alm_iter(f, lmax, lmax, 3)
    res = [_norms(f - oracle.alm2map(a, nside, lmax, lmax)) for a in its]
    for k in range(3):
        assert np.all(res[k + 1] <= res[k] * (1 + 1e-12)), (k, res[k], res[k + 1])


def test_refinement_sign_mistake_is_caught():
    """A planted sign error in the update (a - A r) makes the residual grow:
    the monotone-decrease pin above would fail on it."""
    nside, lmax = 8, 15
    a_true = syn.gaussian_alm(503, lmax, lmax, 1, power=1.0)
    f = oracle.alm2map(a_true, nside, lmax, lmax)
    a = oracle.map2alm(f, lmax, lmax)
    r0 = _norms(f - oracle.alm2map(a, nside, lmax, lmax))
    bad = a - oracle.map2alm(f - oracle.alm2map(a, nside, lmax, lmax), lmax, lmax)
    r1 = _norms(f - oracle.alm2map(bad, nside, lmax, lmax))
    assert np.all(r1 > r0)


# ---------------------------------------------------------------------------
# pixel layouts (Sec. III-B)
# ---------------------------------------------------------------------------
import pytest  # noqa: E402


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32])
def test_layouts_are_bijections_with_exact_centres(nside):
    """Every face pixel's geometric centre is exactly a ring pixel centre of
    Sec. III-A, and the matching is a permutation."""
    perm = oracle.layout_permutations(nside)
    npix = 12 * nside * nside
    for k in ("ring", "nested", "flat"):
        assert np.array_equal(np.sort(perm[k]), np.arange(npix)), k
    z, phi = oracle.face_pixel_centres(nside)
    g = oracle.ring_geometry(nside)
    ring_of_pix = np.repeat(np.arange(4 * nside - 1), g["nphi"])
    r = perm["ring"]
    y = ring_of_pix[r]
    k = r - np.asarray(g["start"])[y]
    zr = np.asarray(g["z"])[y]
    phir = np.pi * (2 * k + np.asarray(g["sigma"])[y]) / np.asarray(g["nphi"])[y]
    assert np.max(np.abs(z - zr)) < 1e-12
    d = np.abs(np.mod(phi - phir + np.pi, 2 * np.pi) - np.pi)
    assert np.max(d) < 1e-12


def test_layout_nside1_is_the_identity():
    assert np.array_equal(oracle.layout_index(1, "ring", "nested"), np.arange(12))


def test_layout_nested_numbering_nside2():
    """The nested numbering of face 0 at Nside 2 (Gorski et al. 2005): its
    pixels 0..3 (south, east, west, north corner) are ring pixels 13, 5, 4, 0.
    Swapping x and y in the Morton interleave (a plausible slip) gives
    13, 4, 5, 0 and fails here."""
    nest2ring = oracle.layout_index(2, "ring", "nested")
    assert list(nest2ring[:4]) == [13, 5, 4, 0]
    assert list(nest2ring[4:8]) == [15, 7, 6, 1]


@pytest.mark.parametrize("nside", [1, 4, 16])
def test_layout_nested_hierarchy(nside):
    """The four children 4p..4p+3 (at 2 nside) of nested pixel p lie around it:
    their mean centre is within a quarter pixel of the parent centre."""
    zp, php = oracle.face_pixel_centres(nside)
    zc, phc = oracle.face_pixel_centres(2 * nside)
    par = oracle.layout_permutations(nside)["nested"]    # flat -> nested
    chi = oracle.layout_permutations(2 * nside)["nested"]
    zpn, ppn = np.empty_like(zp), np.empty_like(php)
    zpn[par], ppn[par] = zp, php
    zcn, pcn = np.empty_like(zc), np.empty_like(phc)
    zcn[chi], pcn[chi] = zc, phc
    zmean = zcn.reshape(-1, 4).mean(axis=1)
    vec = np.exp(1j * pcn.reshape(-1, 4)).mean(axis=1)
    dphi = np.abs(np.angle(vec * np.exp(-1j * ppn)))
    size = np.sqrt(4 * np.pi / (12 * nside * nside))
    sinth = np.sqrt(np.maximum(1 - zpn ** 2, 1e-300))
    assert np.max(np.abs(zmean - zpn)) < 0.25 * size
    assert np.max(dphi * sinth) < 0.25 * size


# ---------------------------------------------------------------------------
# ring quadrature weights (Sec. IV-A)
# ---------------------------------------------------------------------------
from paper_2510_01785_gb300 import weights as hw  # noqa: E402


@pytest.mark.parametrize("nside", [1, 4, 16, 64])
def test_ring_latitudes_match_the_oracle_geometry(nside):
    z, N = hw.ring_latitudes(nside)
    g = oracle.ring_geometry(nside)
    assert np.array_equal(N, g["nphi"])
    assert np.max(np.abs(z - g["z"])) < 1e-15


@pytest.mark.parametrize("nside,lmax", [(4, 8), (16, 32), (16, 47), (64, 128)])
def test_ring_weights_properties(nside, lmax):
    w = hw.ring_weights(nside, lmax)
    z, N = hw.ring_latitudes(nside)
    weq = np.full(4 * nside - 1, 4 * np.pi / (12 * nside * nside))
    assert np.allclose(w, w[::-1], rtol=0, atol=1e-18)                  # north/south symmetric
    assert abs(np.sum(N * w) - 4 * np.pi) < 1e-12                        # total area
    assert hw.quadrature_residual(w, nside, lmax) <= hw.quadrature_residual(weq, nside, lmax)
    assert np.all(np.abs(w / weq - 1) < hw.MAX_DEVIATION)  # the Tikhonov term keeps them near equal


@pytest.mark.parametrize("nside,lmax", [(16, 32), (64, 128)])
def test_ring_weights_improve_band_limited_analysis(nside, lmax):
    a = syn.gaussian_alm(700 + nside, lmax, lmax, 1, power=1.0)
    f = oracle.alm2map(a, nside, lmax, lmax)
    e_eq = np.linalg.norm(oracle.map2alm(f, lmax, lmax) - a)
    e_w = np.linalg.norm(oracle.analysis(f, lmax, lmax, weights=hw.ring_weights(nside, lmax)) - a)
    assert e_w < e_eq


@pytest.mark.parametrize("nside,lmax,gain", [(16, 16, 5.0), (32, 32, 10.0), (32, 48, 4.0), (64, 96, 8.0)])
def test_ring_weights_gain_an_order_of_magnitude_at_low_band_limits(nside, lmax, gain):
    """Where the latitude conditions can be met (lmax up to about 1.5 nside)
    the ring weights cut the analysis error of band-limited maps by about an
    order of magnitude or more (Sec. IV-A reports ~10x for its ring
    weights); the small Tikhonov weight chosen there is what allows it (the
    fixed alpha = 1e-2 gained only 1.5-4x)."""
    a = syn.gaussian_alm(720 + nside, lmax, lmax, 1, power=2.0)
    f = oracle.alm2map(a, nside, lmax, lmax)
    e_eq = np.linalg.norm(oracle.map2alm(f, lmax, lmax) - a)
    e_w = np.linalg.norm(oracle.analysis(f, lmax, lmax, weights=hw.ring_weights(nside, lmax)) - a)
    e_w2 = np.linalg.norm(oracle.analysis(f, lmax, lmax, weights=hw.ring_weights(nside, lmax, alpha=1e-2)) - a)
    assert e_eq / e_w >= gain, e_eq / e_w
    assert e_w < e_w2
