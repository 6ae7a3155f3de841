"""Iterative refinement (Sec. II-A Eq. 4) on the GPU against the oracle's
iterates, step by step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def rel_err(got, ref):
    num = np.linalg.norm((np.atleast_2d(got) - np.atleast_2d(ref)), axis=1)
    return float(np.max(num / np.linalg.norm(np.atleast_2d(ref), axis=1)))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", [(8, 15, 2), (16, 47, 3), (32, 63, 1)])
def test_refinement_matches_oracle(case, dtype):
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = case
    a_true = syn.gaussian_alm(600 + nside, lmax, lmax, nb, power=1.0)
    f = oracle.alm2map(a_true, nside, lmax, lmax)
    rt = np.float64 if dtype == "f64" else np.float32
    f = f.astype(rt).astype(np.float64)
    its = oracle.map2alm_iter(f, lmax, lmax, 3)
    with hpx.Plan(nside, lmax, lmax, nb, dtype) as p:
        df = torch.from_numpy(f.astype(rt)).cuda()
        for k in range(4):
            a = p.map2alm_iter(df, k).cpu().numpy()
            assert rel_err(a, its[k]) <= TOL[dtype], k


def test_refinement_lowers_the_gpu_residual():
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 64, 127, 2
    a_true = torch.from_numpy(syn.gaussian_alm(610, lmax, lmax, nb, power=1.0).astype(np.complex128)).cuda()
    with hpx.Plan(nside, lmax, lmax, nb, "f64") as p:
        f = p.alm2map(a_true)
        res = []
        for k in range(4):
            a = p.map2alm_iter(f, k)
            res.append((f - p.alm2map(a)).norm(dim=1).cpu().numpy())
        for k in range(3):
            assert np.all(res[k + 1] < res[k])
