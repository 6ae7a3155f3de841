"""The seeded input generators: determinism by seed, the stated
distributions, and the coefficient packing, which must agree with the
oracle's own (independently written) index arrays."""
import numpy as np

import oracle
from paper_2510_01785_gb300 import synthetic as syn


def test_same_seed_same_inputs_other_seed_other_inputs():
    a = syn.gaussian_alm(7, 20, 15, 3)
    assert np.array_equal(a, syn.gaussian_alm(7, 20, 15, 3))
    assert not np.array_equal(a, syn.gaussian_alm(8, 20, 15, 3))
    assert np.array_equal(syn.white_maps(3, 4, 2), syn.white_maps(3, 4, 2))
    assert np.array_equal(syn.poisson_arrivals(1, 50.0, 2.0), syn.poisson_arrivals(1, 50.0, 2.0))


def test_packing_matches_the_oracle():
    for lmax, mmax in ((0, 0), (5, 5), (12, 7), (40, 40)):
        ls, ms = oracle.lm_arrays(lmax, mmax)
        assert np.array_equal(syn.packed_l(lmax, mmax), ls)
        assert np.array_equal(syn.packed_m(lmax, mmax), ms)
        assert syn.packed_l(lmax, mmax).size == oracle.nalm(lmax, mmax)
        a = syn.gaussian_alm(1, lmax, mmax, 1)
        assert a.shape == (1, oracle.nalm(lmax, mmax))


def test_gaussian_alm_distribution():
    """Re and Im of a_lm ~ N(0, (l+1)^-p), Im a_l0 = 0: the per-l sample
    variance of (l+1)^(p/2) a_lm over 4000 channels is 1 within 5 sigma."""
    lmax, nb, p = 12, 4000, 2.0
    a = syn.gaussian_alm(11, lmax, lmax, nb, power=p)
    l, m = syn.packed_l(lmax, lmax), syn.packed_m(lmax, lmax)
    assert np.all(a[:, m == 0].imag == 0)
    x = a * (l + 1.0) ** (0.5 * p)
    for ll in range(lmax + 1):
        re = x[:, (l == ll)].real.ravel()
        im = x[:, (l == ll) & (m > 0)].imag.ravel()
        for v in (re, im):
            if v.size:
                assert abs(np.mean(v ** 2) - 1.0) < 5 * np.sqrt(2.0 / v.size), ll
    s = syn.channel_scales(2, nb)
    b = syn.gaussian_alm(11, lmax, lmax, nb, power=p, scales=s)
    assert np.allclose(b, a * s[:, None], rtol=0, atol=0)


def test_white_maps_and_scales():
    w = syn.white_maps(5, 16, 4)
    assert w.shape == (4, 12 * 16 * 16)
    assert abs(w.mean()) < 5 / np.sqrt(w.size) and abs(w.var() - 1) < 5 * np.sqrt(2 / w.size)
    s = syn.channel_scales(9, 1000, 1e-2, 1e3)
    assert s.min() >= 1e-2 and s.max() <= 1e3


def test_poisson_arrivals():
    t = syn.poisson_arrivals(4, 2000.0, 10.0)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] < 10.0
    assert abs(t.size - 20000) < 5 * np.sqrt(20000)
