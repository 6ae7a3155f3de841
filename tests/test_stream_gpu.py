"""Streamed lambda (HPX_PLAN_LAMBDA_STREAM): no table is kept; every
transform refills two staging buffers, block of m by block, with the FP64
recurrence (Eq. 15-16) on a second stream while the tensor cores contract
the other block.  The fill and tile kernels are the resident plan's, so the
results are the resident plan's bit for bit (including several channel
groups per launch and small staging buffers, many blocks per transform); at
Nside 2048, where no table fits, sampled coefficients and rings against the
oracle at the FP32 bar (relative L2 per channel <= 1e-5)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

KINDS = {  # name: (dtype, resident plan keywords)
    "f32-fp16-split": ("f32", dict(lambda_table=True, tensor_cores=True)),
    "f32-tf32x3": ("f32", dict(lambda_table=True, tensor_cores=True, tf32x3=True)),
    "bf16": ("bf16", {}),
    "fp16x3": ("fp16x3", {}),
}


def rel_err(got, ref):
    num = np.linalg.norm((got - ref).reshape(ref.shape[0], -1), axis=1)
    den = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("case", [(64, 191, 191, 3, 1 << 20), (128, 383, 300, 40, 1 << 20), (64, 191, 150, 5, 0)],
                         ids=["ns64-b3-1MiB", "ns128-b40-1MiB", "ns64-b5-default"])
def test_streamed_equals_resident(case, kind):
    import paper_2510_01785_gb300 as hpx
    nside, lmax, mmax, nb, stage = case
    dtype, kw = KINDS[kind]
    maps = torch.from_numpy(syn.white_maps(900 + nside, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(901 + nside, lmax, mmax, nb).astype(np.complex64)).cuda()
    skw = dict(tf32x3=True) if kw.get("tf32x3") else {}
    with hpx.Plan(nside, lmax, mmax, nb, dtype, **kw) as pr, \
            hpx.Plan(nside, lmax, mmax, nb, dtype, streamed=True, stage_bytes=stage, **skw) as ps:
        assert ps.table_bytes == 0 and ps.column_table_bytes == 0 and ps.host_bytes == 0
        if stage:  # (the default staging holds the larger table part twice)
            assert ps.device_bytes < pr.device_bytes
        for op, x in (("map2alm", maps), ("alm2map", alm), ("alm2map_adjoint", maps), ("map2alm_adjoint", alm)):
            a = getattr(pr, op)(x)
            for _ in range(2):  # the staging buffers alternate across calls
                b = getattr(ps, op)(x)
                torch.cuda.synchronize()
                assert torch.equal(a, b), op
        ps.device_status()


def test_streamed_analysis_and_synthesis_interleaved():
    """Both stages on one streamed plan, issued back to back on two streams:
    the staging buffers' events keep every fill behind the last launch that
    read its buffer."""
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 64, 191, 4
    maps = torch.from_numpy(syn.white_maps(910, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(911, lmax, lmax, nb).astype(np.complex64)).cuda()
    with hpx.Plan(nside, lmax, lmax, nb, "f32", lambda_table=True, tensor_cores=True) as pr, \
            hpx.Plan(nside, lmax, lmax, nb, "f32", streamed=True, stage_bytes=1 << 20) as ps:
        ra, rm = pr.map2alm(maps), pr.alm2map(alm)
        torch.cuda.synchronize()
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        outs = []
        for _ in range(3):
            oa, om = ps.empty_alm(), ps.empty_map()
            with torch.cuda.stream(s1):
                ps.map2alm(maps, out=oa)
            with torch.cuda.stream(s2):
                ps.alm2map(alm, out=om)
            outs.append((oa, om))
        torch.cuda.synchronize()
        for oa, om in outs:
            assert torch.equal(oa, ra) and torch.equal(om, rm)
        ps.device_status()


def test_streamed_nside2048_sampled():
    """Nside 2048, lmax 6143, 4 channels (its tables, about 230 GB a part,
    fit nowhere): sampled coefficients at the extreme and aliased m and
    sampled rings at both poles, the last cap ring and the equator, against
    the oracle's separable form."""
    import paper_2510_01785_gb300 as hpx
    ns, lm, nb = 2048, 6143, 4
    maps = syn.white_maps(syn.SEED_BASE + 4, ns, nb).astype(np.float32)
    alm = syn.gaussian_alm(syn.SEED_BASE + 5, lm, lm, nb, power=2.0).astype(np.complex64)
    with hpx.Plan(ns, lm, lm, nb, "f32", streamed=True) as p:
        got_a = p.map2alm(torch.from_numpy(maps).cuda()).cpu().numpy()
        got_s = p.alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
        p.device_status()
    ls, mm = [], []
    r = syn.rng(79)
    for m in (0, 1, 2047, 4095, 4096, 6142, 6143):
        cand = sorted(set([m, min(m + 1, lm), lm] + list(r.integers(m, lm + 1, 3))))
        ls += cand
        mm += [m] * len(cand)
    ls, mm = np.array(ls, np.int32), np.array(mm, np.int32)
    ref = oracle.analysis_sep(maps.astype(np.float64), lm, ls, mm, weights="equal")
    assert rel_err(got_a[:, oracle.alm_index(lm, ls, mm)], ref) <= 1e-5
    R = 4 * ns - 1
    rings = np.array([0, 1, ns - 2, ns - 1, 2 * ns - 1, R - 2, R - 1], np.int32)
    ref_s = oracle.synthesis_sep(alm.astype(np.complex128), ns, lm, lm, rings)
    g = oracle.ring_geometry(ns)
    got = np.concatenate([got_s[:, g["start"][y]: g["start"][y] + g["nphi"][y]] for y in rings], axis=1)
    assert rel_err(got, ref_s) <= 1e-5


def test_streamed_plan_arguments():
    import paper_2510_01785_gb300 as hpx
    with pytest.raises(RuntimeError):  # one m's slice does not fit
        hpx.Plan(64, 191, 191, 1, "f32", streamed=True, stage_bytes=4096)
    with pytest.raises(RuntimeError):  # no tensor-core path for FP64
        hpx.Plan(16, 47, 47, 1, "f64", streamed=True)
    with pytest.raises(ValueError):
        hpx.Plan(16, 47, 47, 1, "f32", streamed=True, out_of_core=True)
