"""Per-ring quadrature weights on the GPU against the oracle's weighted
analysis and weighted synthesis (the analysis adjoint)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn
from paper_2510_01785_gb300 import weights as hw

pytestmark = pytest.mark.gpu


def rel_err(got, ref):
    num = np.linalg.norm(np.atleast_2d(got) - np.atleast_2d(ref), axis=1)
    return float(np.max(num / np.linalg.norm(np.atleast_2d(ref), axis=1)))


@pytest.mark.parametrize("mode,tol", [("f64", 1e-12), ("f32", 1e-5), ("f32tc", 1e-5), ("bf16x3", 1e-4)])
def test_ring_weights_match_oracle(mode, tol):
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 32, 95, 3
    w = hw.ring_weights(nside, lmax)
    rt = np.float64 if mode == "f64" else np.float32
    maps = syn.white_maps(710, nside, nb).astype(rt)
    alm = syn.gaussian_alm(711, lmax, lmax, nb, power=1.0).astype(np.complex128 if mode == "f64" else np.complex64)
    kw = dict(lambda_table=True, tensor_cores=True) if mode == "f32tc" else {}
    dtype = "f32" if mode == "f32tc" else mode
    with hpx.Plan(nside, lmax, lmax, nb, dtype, **kw) as p:
        p.set_ring_weights(w)
        a = p.map2alm(torch.from_numpy(maps).cuda()).cpu().numpy()
        m = p.map2alm_adjoint(torch.from_numpy(alm).cuda()).cpu().numpy()
    ref_a = oracle.analysis(maps.astype(np.float64), lmax, lmax, weights=w)
    ref_m = oracle.synthesis_sep(alm.astype(np.complex128), nside, lmax, lmax, None, w)
    assert rel_err(a, ref_a) <= tol
    assert rel_err(m, ref_m) <= tol


def test_ring_weights_are_validated():
    import paper_2510_01785_gb300 as hpx
    with hpx.Plan(8, 23, 23, 1, "f32") as p:
        with pytest.raises(RuntimeError):
            p.set_ring_weights(np.ones(5))
        bad = np.full(31, 0.1)
        bad[3] = np.nan
        with pytest.raises(RuntimeError):
            p.set_ring_weights(bad)
