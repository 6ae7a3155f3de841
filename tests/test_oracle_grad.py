"""Pin of the gradient convention the GPU's backward passes are checked
against: for real parameters (Re a_lm, Im a_lm) of a real field,

  loss 1  L = sum_l w_l sum_m |a_lm|^2, a = map2alm(p):
          dL/dp = W Y D^-1 (2 w_l a)
  loss 2  L = ||alm2map(a) - t||^2:
          dL/dRe a + i dL/dIm a = D Y^dagger 2 (Y a - t), Im of m = 0 set to 0

with D = 1 for m = 0 and 2 for m >= 1 (Sec. III-F).  Checked against central
finite differences of the oracle's own losses in FP64 on every parameter of
a tiny grid, so a wrong factor of 2 or a missing conjugate fails here.
"""
import numpy as np

import oracle
from paper_2510_01785_gb300 import synthetic as syn

NSIDE, LMAX = 2, 5


def D(lmax):
    _, ms = oracle.lm_arrays(lmax, lmax)
    return np.where(ms == 0, 1.0, 2.0)


def loss1(p, w):
    a = oracle.map2alm(p[None], LMAX, LMAX)[0]
    return float(np.sum(w * np.abs(a) ** 2))


def loss2(a, t):
    return float(np.sum((oracle.alm2map(a[None], NSIDE, LMAX, LMAX)[0] - t) ** 2))


def test_loss1_gradient_formula_matches_finite_differences():
    ls, _ = oracle.lm_arrays(LMAX, LMAX)
    w = 1.0 / (ls + 1.0)
    p = syn.white_maps(41, NSIDE, 1)[0]
    a = oracle.map2alm(p[None], LMAX, LMAX)[0]
    grad = oracle.map2alm_adjoint(((2 * w * a) / D(LMAX))[None], NSIDE, LMAX, LMAX)[0]
    h = 1e-5
    fd = np.zeros_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (loss1(p + e, w) - loss1(p - e, w)) / (2 * h)
    assert np.max(np.abs(fd - grad)) < 1e-8 * np.max(np.abs(grad))


def test_loss2_gradient_formula_matches_finite_differences():
    _, ms = oracle.lm_arrays(LMAX, LMAX)
    a = syn.gaussian_alm(42, LMAX, LMAX, 1, power=0.0)[0]
    t = syn.white_maps(43, NSIDE, 1)[0]
    r = oracle.alm2map(a[None], NSIDE, LMAX, LMAX)[0] - t
    grad = D(LMAX) * oracle.alm2map_adjoint((2 * r)[None], LMAX, LMAX)[0]
    grad = np.where(ms == 0, grad.real + 0j, grad)
    h = 1e-6
    fd = np.zeros_like(a)
    for k in range(a.size):
        for part, unit in ((0, 1.0), (1, 1j)):
            e = np.zeros_like(a)
            e[k] = h * unit
            d = (loss2(a + e, t) - loss2(a - e, t)) / (2 * h)
            fd[k] += d if part == 0 else 1j * d
    assert np.max(np.abs(fd - grad)) < 1e-8 * np.max(np.abs(grad))
    assert np.all(fd[ms == 0].imag == 0.0) or np.max(np.abs(fd[ms == 0].imag)) < 1e-9
