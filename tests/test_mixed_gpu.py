"""Mixed-precision dtypes (16-bit lambda tables and operands on the tensor
cores, FP32 accumulation) against the FP64 oracle.

Inputs follow the mixed-precision workload: coefficients with variance
(l+1)^-3 and maps of white noise, each channel scaled by a factor drawn
uniformly from [1e-2, 1e3], so one channel cannot hide another and the FP16
channel scaling is exercised across five decades.

Bounds (relative L2 per channel, worst channel), from the expected rounding
of each mode: BF16 keeps 8 significant bits (2^-9 = 2e-3 per operand), FP16
11 (2^-12 = 2.4e-4), and the x3 split products keep about twice as many.
  bf16 <= 1e-2, bf16x3 <= 1e-4, fp16 <= 2e-3, fp16x3 <= 1e-5
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

BOUND = {"bf16": 1e-2, "bf16x3": 1e-4, "fp16": 2e-3, "fp16x3": 1e-5}


def hpx():
    import paper_2510_01785_gb300 as h
    return h


def rel_err(got, ref):
    got = np.atleast_2d(np.asarray(got))
    ref = np.atleast_2d(np.asarray(ref))
    num = np.linalg.norm((got - ref).reshape(ref.shape[0], -1), axis=1)
    den = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


CASES = [
    # nside, lmax, mmax, nbatch
    (2, 5, 5, 3),
    (8, 23, 23, 3),
    (16, 47, 20, 5),        # mmax < lmax
    (32, 95, 95, 17),       # 32 channels per launch
    (64, 191, 191, 40),     # analysis 64 per launch; synthesis two launches
    (128, 383, 383, 2),
    (256, 767, 767, 3),
]


@pytest.fixture(scope="module")
def refs():
    cache = {}

    def get(case):
        if case not in cache:
            nside, lmax, mmax, nb = case
            sc = syn.channel_scales(syn.SEED_BASE + 30 + nside, nb)
            maps = (syn.white_maps(syn.SEED_BASE + 31 + nside, nside, nb) * sc[:, None]).astype(np.float32)
            alm = syn.gaussian_alm(syn.SEED_BASE + 32 + nside, lmax, mmax, nb, power=3.0,
                                   scales=sc).astype(np.complex64)
            m64, a64 = maps.astype(np.float64), alm.astype(np.complex128)
            cache[case] = dict(
                maps=maps, alm=alm,
                map2alm=oracle.map2alm(m64, lmax, mmax),
                alm2map=oracle.alm2map(a64, nside, lmax, mmax),
                alm2map_adjoint=oracle.alm2map_adjoint(m64, lmax, mmax),
                map2alm_adjoint=oracle.map2alm_adjoint(a64, nside, lmax, mmax))
        return cache[case]
    return get


@pytest.mark.parametrize("mode", list(BOUND))
@pytest.mark.parametrize("case", CASES, ids=[f"ns{c[0]}-l{c[1]}-m{c[2]}-b{c[3]}" for c in CASES])
def test_mixed_parity(case, mode, refs):
    nside, lmax, mmax, nb = case
    r = refs(case)
    with hpx().Plan(nside, lmax, mmax, nb, mode) as p:
        dm, da = torch.from_numpy(r["maps"]).cuda(), torch.from_numpy(r["alm"]).cuda()
        got = {"map2alm": p.map2alm(dm), "alm2map_adjoint": p.alm2map_adjoint(dm),
               "alm2map": p.alm2map(da), "map2alm_adjoint": p.map2alm_adjoint(da)}
        p.device_status()
        for k, v in got.items():
            e = rel_err(v.cpu().numpy(), r[k])
            print(f"{mode} {case} {k}: {e:.3e}")
            assert e <= BOUND[mode], (k, e)
        a = got["map2alm"].cpu().numpy()
        assert np.all(a[:, : lmax + 1].imag == 0.0)


def test_mixed_tables_are_smaller():
    """Single 16-bit tables take half the FP32 table's bytes; x3 the same."""
    h = hpx()
    with h.Plan(64, 191, 191, 2, "f32", lambda_table=True, tensor_cores=True) as pf, \
            h.Plan(64, 191, 191, 2, "bf16") as pb, h.Plan(64, 191, 191, 2, "fp16x3") as px:
        assert 0 < pb.table_bytes < 0.6 * pf.table_bytes
        assert 0 < pb.column_table_bytes < 0.6 * pf.column_table_bytes
        assert px.table_bytes > 1.5 * pb.table_bytes


def test_mixed_deterministic():
    nside, lmax, nb = 64, 191, 5
    maps = torch.from_numpy(syn.white_maps(94, nside, nb).astype(np.float32)).cuda()
    for mode in BOUND:
        with hpx().Plan(nside, lmax, lmax, nb, mode) as p:
            a1 = p.map2alm(maps).clone()
            s1 = p.alm2map(a1).clone()
            assert torch.equal(p.map2alm(maps), a1) and torch.equal(p.alm2map(a1), s1)
            p.device_status()


NS3, L3, B3 = 1024, 2047, 64


@pytest.fixture(scope="module")
def cfg3():
    """The mixed-precision workload at full size: 64 channels scaled over
    [1e-2, 1e3], coefficients of variance (l+1)^-3 and white-noise maps (both
    from the seeded generators; no input comes from the GPU path), and the
    oracle's values of three channels (the smallest and largest scales and
    one between) on sampled coefficients and rings."""
    sc = syn.channel_scales(syn.SEED_BASE + 33, B3)
    alm = syn.gaussian_alm(syn.SEED_BASE + 34, L3, L3, B3, power=3.0, scales=sc)
    maps = (syn.white_maps(syn.SEED_BASE + 35, NS3, B3) * sc[:, None]).astype(np.float32).astype(np.float64)
    alm = alm.astype(np.complex64).astype(np.complex128)
    chans = [int(np.argmin(sc)), int(np.argmax(sc)), 17]
    r = syn.rng(79)
    ms = [0, 1, 2, 127, 128, 1000, 1500, 2046, 2047]
    ls, mm = [], []
    for m in ms:
        cand = sorted(set([m, min(m + 1, L3), min(m + 63, L3), min(m + 64, L3), L3] + list(r.integers(m, L3 + 1, 3))))
        ls += cand
        mm += [m] * len(cand)
    ls, mm = np.array(ls, np.int32), np.array(mm, np.int32)
    rings = np.array([0, 1, 2, 127, 1023, 2047, 3070, 4 * NS3 - 3, 4 * NS3 - 2], np.int32)
    ref_a = oracle.analysis_sep(maps[chans], L3, ls, mm, weights="equal")
    ref_m = oracle.synthesis_sep(alm[chans], NS3, L3, L3, rings)
    return dict(maps=maps.astype(np.float32), alm=alm.astype(np.complex64), chans=chans, ls=ls, mm=mm,
                rings=rings, ref_a=ref_a, ref_m=ref_m)


@pytest.mark.parametrize("mode", ["f32"] + list(BOUND))
def test_cfg3_full_size_sampled(mode, cfg3):
    """Nside 1024, lmax 2047, 64 channels, in the launch configuration the
    benchmark times: sampled coefficients and rings of three channels against
    the oracle, each mode within its bound (FP32: 1e-5)."""
    h = hpx()
    kw = dict(lambda_table=True, tensor_cores=True) if mode == "f32" else {}
    with h.Plan(NS3, L3, L3, B3, mode, **kw) as p:
        a = p.map2alm(torch.from_numpy(cfg3["maps"]).cuda())
        s = p.alm2map(torch.from_numpy(cfg3["alm"]).cuda())
        p.device_status()
        a, s = a.cpu().numpy(), s.cpu().numpy()
    c = cfg3["chans"]
    ea = rel_err(a[c][:, oracle.alm_index(L3, cfg3["ls"], cfg3["mm"])], cfg3["ref_a"])
    g = oracle.ring_geometry(NS3)
    got = np.concatenate([s[c][:, g["start"][y]: g["start"][y] + g["nphi"][y]] for y in cfg3["rings"]], axis=1)
    es = rel_err(got, cfg3["ref_m"])
    bound = 1e-5 if mode == "f32" else BOUND[mode]
    print(f"cfg3 {mode}: analysis {ea:.3e}, synthesis {es:.3e}")
    assert ea <= bound and es <= bound, (ea, es)
