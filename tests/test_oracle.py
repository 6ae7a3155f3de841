"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these checks retypes the oracle's own formulas: each compares it with
an independent source -- a textbook library routine (scipy's spherical
harmonics, numpy's Legendre series and FFT), a closed form, an identity the
grid or the harmonics must satisfy, an exact symmetry of the grid, or a brute
force sum over pixel centres.
"""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y

import oracle
from paper_2510_01785_gb300 import synthetic as syn


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# --------------------------------------------------------------------------
# geometry (Sec. III-A)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nside", [1, 2, 4, 8, 64, 1024])
def test_geometry_counts_and_prefix(nside):
    g = oracle.ring_geometry(nside)
    R = 4 * nside - 1
    assert g["nphi"].shape == (R,)
    assert int(g["nphi"].sum()) == 12 * nside * nside
    # start pixels are the prefix sums of the ring lengths (RING order)
    assert np.array_equal(g["start"], np.concatenate([[0], np.cumsum(g["nphi"])[:-1]]))
    # 4 pixels next to the poles, 4 Nside on the equatorial rings (Sec. III-A)
    assert g["nphi"][0] == 4 and g["nphi"][-1] == 4
    assert g["nphi"].max() == 4 * nside
    assert np.all(g["nphi"] % 4 == 0)


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 256, 2048])
def test_geometry_equal_area(nside):
    """Equal-area pixels: the spherical cap above ring y's centre holds
    exactly start_y + N_y / 2 pixel areas of 4 pi / Npix."""
    g = oracle.ring_geometry(nside)
    npix = 12 * nside * nside
    cap = 2 * np.pi * (1 - g["z"])
    pixels = (g["start"] + g["nphi"] / 2) * 4 * np.pi / npix
    assert np.max(np.abs(cap - pixels)) < 1e-13


@pytest.mark.parametrize("nside", [1, 2, 8, 512])
def test_geometry_mirror_and_unit_circle(nside):
    g = oracle.ring_geometry(nside)
    assert np.allclose(g["z"], -g["z"][::-1], atol=0, rtol=1e-15)
    assert np.array_equal(g["nphi"], g["nphi"][::-1])
    assert np.array_equal(g["sigma"], g["sigma"][::-1])
    assert np.max(np.abs(g["z"] ** 2 + g["sinth"] ** 2 - 1)) < 1e-15
    assert np.all(np.diff(g["z"]) < 0)  # north to south


def test_geometry_known_pixel_centres():
    """Hand-derived HEALPix pixel centres: at Nside 1 the rings sit at
    z = 2/3, 0, -2/3 with the middle ring starting at phi = 0 and the others
    at pi/4; at Nside 2 the first ring is at z = 11/12, ring 3 at 1/3 with no
    half-pixel shift."""
    g1 = oracle.ring_geometry(1)
    assert np.allclose(g1["z"], [2 / 3, 0, -2 / 3], rtol=0, atol=1e-16)
    assert list(g1["sigma"]) == [1, 0, 1]
    th, ph = oracle.pixel_angles(1)
    assert ph[0] == pytest.approx(np.pi / 4) and ph[4] == 0.0
    g2 = oracle.ring_geometry(2)
    assert g2["z"][0] == pytest.approx(11 / 12, abs=1e-16)
    assert g2["z"][2] == pytest.approx(1 / 3, abs=1e-16)
    assert list(g2["sigma"]) == [1, 1, 0, 1, 0, 1, 1]
    assert list(g2["nphi"]) == [4, 8, 8, 8, 8, 8, 4]


# --------------------------------------------------------------------------
# lambda_lm (Eq. 8, 15, 16)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("theta", [0.013, 0.4, 1.1, np.pi / 2, 2.3, 3.1])
def test_lambda_vs_scipy(theta):
    lmax = 60
    z, s = np.cos(theta), np.sin(theta)
    for m in range(0, lmax + 1, 3):
        ours = oracle.lambda_chain(lmax, m, z, s)
        ref = np.real(sph_harm_y(np.arange(m, lmax + 1), m, theta, 0.0))
        scale = np.max(np.abs(ref)) + 1e-300
        assert np.max(np.abs(ours - ref)) <= 1e-12 * scale, (m, theta)


def test_lambda_closed_forms():
    for theta in [0.2, 1.0, 2.5]:
        z, s = np.cos(theta), np.sin(theta)
        l0 = oracle.lambda_chain(2, 0, z, s)
        l1 = oracle.lambda_chain(2, 1, z, s)
        l2 = oracle.lambda_chain(2, 2, z, s)
        assert l0[0] == pytest.approx(1 / np.sqrt(4 * np.pi), rel=1e-15)
        assert l0[1] == pytest.approx(np.sqrt(3 / (4 * np.pi)) * z, rel=1e-14)
        assert l0[2] == pytest.approx(np.sqrt(5 / (16 * np.pi)) * (3 * z * z - 1), rel=1e-13)
        # Condon-Shortley phase: Y_11 = -sqrt(3/8pi) sin(theta) e^{i phi}
        assert l1[0] == pytest.approx(-np.sqrt(3 / (8 * np.pi)) * s, rel=1e-14)
        assert l1[1] == pytest.approx(-np.sqrt(15 / (8 * np.pi)) * s * z, rel=1e-14)
        assert l2[0] == pytest.approx(np.sqrt(15 / (32 * np.pi)) * s * s, rel=1e-14)


def test_lambda_m0_is_legendre():
    lmax = 300
    for z in [-0.97, -0.3, 0.0, 0.51, 0.999]:
        ours = oracle.lambda_chain(lmax, 0, z, np.sqrt(1 - z * z))
        ref = np.array([np.sqrt((2 * l + 1) / (4 * np.pi)) *
                        np.polynomial.legendre.legval(z, [0] * l + [1]) for l in range(lmax + 1)])
        assert np.max(np.abs(ours - ref)) < 1e-12


@pytest.mark.parametrize("nside,which", [(2048, 0), (2048, 2047), (2048, 4095), (64, 5)])
def test_lambda_addition_theorem_high_l(nside, which):
    """sum_m |Y_lm|^2 = (2l+1)/4pi at every theta: lambda_l0^2 + 2 sum_{m>=1}
    lambda_lm^2 = (2l+1)/4pi.  At lmax = 3*2048-1 on the first ring of
    Nside 2048 most chains start far below the double range, so this pins the
    rescaled recursion at high l.  sin(theta) is taken as sqrt((1-z)(1+z))
    of the stored z so the pair lies on the unit circle to rounding: near the
    pole a double z carries only ~1e-9 relative precision in 1 - z, and the
    identity is sensitive to that, not to the recursion."""
    lmax = 3 * nside - 1
    g = oracle.ring_geometry(nside)
    z = g["z"][which]
    s = np.sqrt((1.0 - z) * (1.0 + z))
    tot = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        lam = oracle.lambda_chain(lmax, m, z, s)
        tot[m:] += (1.0 if m == 0 else 2.0) * lam ** 2
    ref = (2 * np.arange(lmax + 1) + 1) / (4 * np.pi)
    # near the pole the recurrence behaves like x_l = 2 x_{l-1} - x_{l-2},
    # whose rounding errors grow like l^1.5 eps: bound 1e-15 (l+1)^1.5
    bound = 1e-15 * (np.arange(lmax + 1) + 1.0) ** 1.5
    assert np.all(np.abs(tot / ref - 1) < bound)


def test_lambda_mm_deep_underflow_log():
    """log2|lambda_mm| = log2 sqrt(Gamma(m+3/2) / (4 pi Gamma(3/2) Gamma(m+1)))
    + m log2 sin(theta), far below the double range."""
    for m, s in [(6143, 4.0e-4), (3071, 7.97e-4), (500, 0.3)]:
        z = np.sqrt(1 - s * s)
        lg, sg = oracle.lambda_chain_log2(m, m, z, s)
        ref = 0.5 * (math.lgamma(m + 1.5) - math.lgamma(1.5) - math.lgamma(m + 1)
                     - math.log(4 * math.pi)) / math.log(2) + m * math.log2(s)
        assert abs(lg[0] - ref) < 1e-9 * max(1.0, abs(ref))
        assert sg[0] == (-1.0) ** m


def test_lambda_log_chain_matches_double_chain():
    """Where lambda is representable both outputs of the recursion agree;
    where it is not, the double output is exactly zero."""
    lmax, m, s = 3071, 1800, 0.65
    z = np.sqrt(1 - s * s)
    v = oracle.lambda_chain(lmax, m, z, s)
    lg, sg = oracle.lambda_chain_log2(lmax, m, z, s)
    ok = lg > -1000
    assert np.any(ok) and np.any(~ok)
    assert np.allclose(np.log2(np.abs(v[ok])), lg[ok], rtol=0, atol=1e-12)
    assert np.all(np.sign(v[ok]) == sg[ok])
    assert np.all(np.abs(v[lg < -1080]) == 0.0)


# --------------------------------------------------------------------------
# ring DFT and the aliasing fold (Eq. 13, Eq. 26)
# --------------------------------------------------------------------------
def test_ring_modes_vs_numpy_fft():
    r = syn.rng(11)
    for n in [4, 8, 12, 20, 28, 64]:
        for sigma in [0, 1]:
            p = r.standard_normal(n)
            ms = np.arange(0, 3 * n + 5, dtype=np.int32)
            G = oracle.ring_modes(p, sigma, ms)
            F = np.fft.fft(p)
            ref = F[ms % n] * np.exp(-1j * np.pi * sigma * ms / n)
            assert np.max(np.abs(G - ref)) < 1e-13 * n


def test_single_mode_synthesis_recovers_lambda():
    """A one-hot a_lm with 2m < N_y synthesises to a ring whose m-th Fourier
    sum is N_y a_lm lambda_lm(z_y) (DFT orthogonality)."""
    nside, lmax, mmax = 4, 11, 11
    g = oracle.ring_geometry(nside)
    n_alm = oracle.nalm(lmax, mmax)
    for (l, m) in [(3, 1), (7, 2), (11, 5)]:
        a = np.zeros((1, n_alm), np.complex128)
        a[0, oracle.alm_index(lmax, l, m)] = 0.7 - 0.4j
        p = oracle.alm2map(a, nside, lmax, mmax)[0]
        for y in range(4 * nside - 1):
            n = int(g["nphi"][y])
            if 2 * m >= n:
                continue
            ring = p[g["start"][y]: g["start"][y] + n]
            G = oracle.ring_modes(ring, int(g["sigma"][y]), [m])[0]
            lam = oracle.lambda_chain(l, m, g["z"][y], g["sinth"][y])[-1]
            assert abs(G - n * (0.7 - 0.4j) * lam) < 1e-13


# --------------------------------------------------------------------------
# the operators against brute force over pixel centres with scipy's Y_lm
# --------------------------------------------------------------------------
def scipy_Y(nside, lmax, mmax):
    th, ph = oracle.pixel_angles(nside)
    ls, ms = oracle.lm_arrays(lmax, mmax)
    return sph_harm_y(ls[:, None], ms[:, None], th[None, :], ph[None, :])  # [nalm, npix]


@pytest.mark.parametrize("nside,lmax", [(1, 2), (2, 5), (2, 9), (4, 11), (4, 17)])
def test_analysis_vs_scipy_brute_force(nside, lmax):
    """Eq. 1: a_lm = (4 pi / N) sum_i conj(Y_lm(theta_i, phi_i)) f_i, with
    scipy's Y_lm.  lmax >= N_y covers the aliased m of the polar rings."""
    mmax = lmax
    Y = scipy_Y(nside, lmax, mmax)
    f = syn.white_maps(3, nside, 2)
    ref = (4 * np.pi / f.shape[1]) * (f @ np.conj(Y).T)
    for tier in ["direct", "sep"]:
        got = oracle.map2alm(f, lmax, mmax, tier=tier)
        assert np.max(np.abs(got - ref)) < 1e-13, tier


@pytest.mark.parametrize("nside,lmax,mmax", [(1, 2, 2), (2, 5, 5), (2, 9, 4), (4, 11, 11)])
def test_synthesis_vs_scipy_brute_force(nside, lmax, mmax):
    """Eq. 2: f_i = sum_l sum_{m=-l..l} a_lm Y_lm(theta_i, phi_i), with
    a_{l,-m} = (-1)^m conj(a_lm) for a real field, using scipy's Y_lm."""
    Y = scipy_Y(nside, lmax, mmax)
    ls, ms = oracle.lm_arrays(lmax, mmax)
    a = syn.gaussian_alm(5, lmax, mmax, 2, power=0.0)
    # sum over m >= 0 plus the mirrored -m terms: Y_{l,-m} = (-1)^m conj(Y_lm)
    pos = a @ Y
    neg = (np.where(ms > 0, 1.0, 0.0) * np.conj(a)) @ np.conj(Y)
    ref = pos + neg
    assert np.max(np.abs(ref.imag)) < 1e-12
    for tier in ["direct", "sep"]:
        got = oracle.alm2map(a, nside, lmax, mmax, tier=tier)
        assert np.max(np.abs(got - ref.real)) < 1e-12, tier


@pytest.mark.parametrize("nside", [2, 4, 8])
def test_tier_a_equals_tier_b(nside):
    lmax = 3 * nside - 1
    mmax = lmax - 1
    f = syn.white_maps(7, nside, 2)
    a = syn.gaussian_alm(8, lmax, mmax, 2)
    A = oracle.map2alm(f, lmax, mmax, tier="direct")
    B = oracle.map2alm(f, lmax, mmax, tier="sep")
    assert rel(A, B) < 1e-14
    P = oracle.alm2map(a, nside, lmax, mmax, tier="direct")
    Q = oracle.alm2map(a, nside, lmax, mmax, tier="sep")
    assert rel(P, Q) < 1e-14


# --------------------------------------------------------------------------
# exact properties of the grid and the operators
# --------------------------------------------------------------------------
def test_constant_map():
    nside, lmax = 8, 23
    f = np.ones((1, 12 * nside * nside))
    a = oracle.map2alm(f, lmax, lmax)[0]
    ls, ms = oracle.lm_arrays(lmax, lmax)
    assert a[0] == pytest.approx(np.sqrt(4 * np.pi), rel=1e-14)
    assert np.max(np.abs(a[(ms == 0) & (ls % 2 == 1)])) < 1e-14
    assert np.max(np.abs(a[ms % 4 != 0])) < 1e-14


def test_real_input_gives_real_m0():
    f = syn.white_maps(9, 4, 3)
    a = oracle.map2alm(f, 11, 11)
    _, ms = oracle.lm_arrays(11, 11)
    assert np.all(a[:, ms == 0].imag == 0.0)


def test_rotation_by_quarter_turn():
    """Rolling every ring by N_y/4 pixels rotates the sphere by pi/2 about the
    axis (a grid symmetry): a_lm -> a_lm exp(-i m pi/2)."""
    nside, lmax = 4, 11
    g = oracle.ring_geometry(nside)
    f = syn.white_maps(12, nside, 1)
    fr = f.copy()
    for y in range(4 * nside - 1):
        s, n = g["start"][y], g["nphi"][y]
        fr[0, s:s + n] = np.roll(f[0, s:s + n], n // 4)
    a = oracle.map2alm(f, lmax, lmax)
    ar = oracle.map2alm(fr, lmax, lmax)
    _, ms = oracle.lm_arrays(lmax, lmax)
    assert rel(ar, a * np.exp(-0.5j * np.pi * ms)) < 1e-14


def test_north_south_reflection():
    """Swapping ring y with ring R-1-y reflects z: a_lm -> (-1)^(l+m) a_lm."""
    nside, lmax = 4, 11
    g = oracle.ring_geometry(nside)
    R = 4 * nside - 1
    f = syn.white_maps(13, nside, 1)
    fr = np.zeros_like(f)
    for y in range(R):
        s, n = g["start"][y], g["nphi"][y]
        s2 = g["start"][R - 1 - y]
        fr[0, s:s + n] = f[0, s2:s2 + n]
    a = oracle.map2alm(f, lmax, lmax)
    ar = oracle.map2alm(fr, lmax, lmax)
    ls, ms = oracle.lm_arrays(lmax, lmax)
    assert rel(ar, a * (-1.0) ** (ls + ms)) < 1e-14


@pytest.mark.parametrize("nside", [2, 4, 8])
def test_adjoint_identities(nside):
    """Sec. III-F: <Y a, p> = <a, Y^dagger p>_full and
    <A p, a>_full = <p, W Y a>, A = Y^dagger W; with equal weights
    A = (4 pi / Npix) Y^dagger."""
    lmax = 3 * nside - 1
    mmax = lmax
    p = syn.white_maps(21, nside, 1)
    a = syn.gaussian_alm(22, lmax, mmax, 1, power=0.0)
    Ya = oracle.alm2map(a, nside, lmax, mmax)
    Ytp = oracle.alm2map_adjoint(p, lmax, mmax)
    lhs, rhs = float(np.sum(Ya * p)), oracle.inner_full(a, Ytp, lmax, mmax)
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1)
    Ap = oracle.map2alm(p, lmax, mmax)
    WYa = oracle.map2alm_adjoint(a, nside, lmax, mmax)
    lhs, rhs = oracle.inner_full(Ap, a, lmax, mmax), float(np.sum(p * WYa))
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1)
    assert rel(Ap, (4 * np.pi / p.shape[1]) * Ytp) < 1e-15


def test_quadrature_accuracy_improves_with_nside():
    """A single low-l mode synthesised and analysed again comes back to
    quadrature accuracy, better at every finer grid (Sec. IV-A)."""
    errs = []
    for nside in [2, 4, 8, 16]:
        lmax = 4
        n_alm = oracle.nalm(lmax, lmax)
        a = np.zeros((1, n_alm), np.complex128)
        a[0, oracle.alm_index(lmax, 1, 0)] = 1.0  # Y_10 ∝ cos(theta)
        a[0, oracle.alm_index(lmax, 3, 2)] = 0.5 - 0.25j
        f = oracle.alm2map(a, nside, lmax, lmax)
        back = oracle.map2alm(f, lmax, lmax)
        errs.append(np.max(np.abs(back - a)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-3 and errs[0] < 0.2, errs
