"""Tensor-core (tcgen05) Legendre stages of the FP32 plan, in both split
schemes (FP16 hi/lo, the default, and 3xTF32), against the FP64 oracle and
against the CUDA-core path on the same table.

The tensor-core plan computes the same sums as the CUDA-core FP32 path, in a
different order and from split products, so it is held to the FP32
tolerance against the oracle (relative L2 per channel <= 1e-5) and its
error may not exceed twice that of the CUDA-core FP32 path (plus 1e-6).
Cases cover every N tile (8, 16 and 32 channels per launch), more channels
than one launch takes,
tiles that end past lmax, mmax < lmax, and groups whose rows start inside
the l range.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


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
    (1, 2, 2, 1),
    (2, 5, 5, 3),
    (8, 40, 30, 2),        # every ring aliases
    (16, 47, 20, 3),       # mmax < lmax
    (32, 0, 0, 1),         # lmax = 0
    (64, 191, 191, 9),     # N = 64 (16 channels per launch), ragged
    (32, 95, 95, 17),      # N = 128, ragged
    (32, 95, 95, 40),      # two launches (32 + 8 channels)
    (32, 95, 95, 70),      # three launches (32 + 32 + 6)
    (128, 383, 383, 2),    # three l tiles per low m
    (256, 400, 380, 1),
    (512, 1535, 1535, 2),  # group starts well inside the l range
]


SCHEMES = {"fp16-split": False, "tf32x3": True}


@pytest.mark.parametrize("scheme", list(SCHEMES))
@pytest.mark.parametrize("case", CASES, ids=[f"ns{c[0]}-l{c[1]}-m{c[2]}-b{c[3]}" for c in CASES])
def test_tensor_core_parity(case, scheme):
    nside, lmax, mmax, nb = case
    maps = syn.white_maps(syn.SEED_BASE + 300 + nside, nside, nb).astype(np.float32)
    alm = syn.gaussian_alm(syn.SEED_BASE + 400 + nside, lmax, mmax, nb, power=1.0).astype(np.complex64)
    m64, a64 = maps.astype(np.float64), alm.astype(np.complex128)
    h = hpx()
    with h.Plan(nside, lmax, mmax, nb, "f32", lambda_table=True, tensor_cores=True,
                tf32x3=SCHEMES[scheme]) as pc, \
            h.Plan(nside, lmax, mmax, nb, "f32", lambda_table=True) as pt:
        dm, da = torch.from_numpy(maps).cuda(), torch.from_numpy(alm).cuda()
        ops = (("map2alm", dm), ("alm2map_adjoint", dm), ("alm2map", da), ("map2alm_adjoint", da))
        got = {k: getattr(pc, k)(x) for k, x in ops}
        cuda_core = {k: getattr(pt, k)(x) for k, x in ops}
        pc.device_status()
        ref = {"map2alm": oracle.map2alm(m64, lmax, mmax),
               "alm2map_adjoint": oracle.alm2map_adjoint(m64, lmax, mmax),
               "alm2map": oracle.alm2map(a64, nside, lmax, mmax),
               "map2alm_adjoint": oracle.map2alm_adjoint(a64, nside, lmax, mmax)}
        for k, v in got.items():
            e = rel_err(v.cpu().numpy(), ref[k])
            assert e <= 1e-5, (k, e)
            if k in cuda_core:  # no worse than the CUDA-core FP32 path, up to rounding noise
                e_cc = rel_err(cuda_core[k].cpu().numpy(), ref[k])
                print(f"{case} {k}: tensor cores {e:.3e}, CUDA cores {e_cc:.3e}")
                assert e <= 2.0 * e_cc + 1e-6, (k, e, e_cc)
        a = got["map2alm"].cpu().numpy()
        assert np.all(a[:, : lmax + 1].imag == 0.0)


@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_tensor_core_dynamic_range(scheme):
    """Channels scaled by 1e-30 .. 1e30 (FP32's range; far outside FP16's):
    every channel keeps the FP32 tolerance, so the per-channel power-of-two
    scaling of the 16-bit operands covers the whole float range."""
    nside, lmax, nb = 32, 95, 7
    sc = np.array([1e-30, 1e-12, 1e-3, 1.0, 1e5, 1e18, 1e30])
    maps = (syn.white_maps(syn.SEED_BASE + 61, nside, nb) * sc[:, None]).astype(np.float32)
    alm = (syn.gaussian_alm(syn.SEED_BASE + 62, lmax, lmax, nb, power=2.0) * sc[:, None]).astype(np.complex64)
    with hpx().Plan(nside, lmax, lmax, nb, "f32", lambda_table=True, tensor_cores=True,
                    tf32x3=SCHEMES[scheme]) as pc:
        a = pc.map2alm(torch.from_numpy(maps).cuda()).cpu().numpy()
        s = pc.alm2map(torch.from_numpy(alm).cuda()).cpu().numpy()
        pc.device_status()
    ea = rel_err(a, oracle.map2alm(maps.astype(np.float64), lmax, lmax))
    es = rel_err(s, oracle.alm2map(alm.astype(np.complex128), nside, lmax, lmax))
    print(scheme, ea, es)
    assert ea <= 1e-5 and es <= 1e-5


def test_tensor_core_gradient_scaling():
    """The gradient entry points (m > 0 doubled on the way out of the
    analysis, halved on the way into the synthesis) run through the same tile
    kernels: they match the CUDA-core table plan."""
    nside, lmax, nb = 64, 191, 3
    maps = torch.from_numpy(syn.white_maps(91, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(93, lmax, lmax, nb).astype(np.complex64)).cuda()
    h = hpx()
    with h.Plan(nside, lmax, lmax, nb, "f32", lambda_table=True, tensor_cores=True) as pc, \
            h.Plan(nside, lmax, lmax, nb, "f32", lambda_table=True) as pt:
        for op, x in (("alm2map_grad", maps), ("map2alm_grad", alm)):
            g1 = getattr(pc, op)(x)
            g2 = getattr(pt, op)(x)
            torch.cuda.synchronize()
            assert rel_err(g1.cpu().numpy(), g2.cpu().numpy()) <= 1e-5, op


def test_tensor_core_deterministic_and_status():
    nside, lmax, nb = 128, 383, 5
    maps = torch.from_numpy(syn.white_maps(92, nside, nb).astype(np.float32)).cuda()
    with hpx().Plan(nside, lmax, lmax, nb, "f32", lambda_table=True, tensor_cores=True) as pc:
        a1 = pc.map2alm(maps).clone()
        a2 = pc.map2alm(maps)
        s1 = pc.alm2map(a1).clone()
        s2 = pc.alm2map(a1)
        pc.device_status()
        assert torch.equal(a1, a2) and torch.equal(s1, s2)
        host = pc.map2alm_host(maps.cpu().numpy())
        assert np.array_equal(host.numpy(), a1.cpu().numpy())
        host = pc.alm2map_host(a1.cpu().numpy())
        assert np.array_equal(host.numpy(), s1.cpu().numpy())


NS2, L2, B2 = 1024, 3071, 8


def test_cfg2_tensor_core_sampled():
    """Nside 1024, lmax 3071, 8 channels (the default FP16 hi/lo scheme, as
    benchmarked): sampled coefficients and rings against the oracle, and
    whole outputs against the CUDA-core table plan."""
    maps = syn.white_maps(syn.SEED_BASE + 2, NS2, B2).astype(np.float32)
    alm_in = syn.gaussian_alm(syn.SEED_BASE + 3, L2, L2, B2, power=2.0).astype(np.complex64)
    h = hpx()
    dm, da = torch.from_numpy(maps).cuda(), torch.from_numpy(alm_in).cuda()
    with h.Plan(NS2, L2, L2, B2, "f32", lambda_table=True, tensor_cores=True) as pc:
        a = pc.map2alm(dm)
        smap = pc.alm2map(da)
        pc.device_status()
        a, smap = a.cpu().numpy(), smap.cpu().numpy()
    with h.Plan(NS2, L2, L2, B2, "f32", lambda_table=True) as pt:
        b = pt.map2alm(dm).cpu().numpy()
        bmap = pt.alm2map(da).cpu().numpy()
    assert rel_err(a, b) <= 1e-5
    assert rel_err(smap, bmap) <= 1e-5
    R = 4 * NS2 - 1
    rings = np.array([0, 1, 2, 127, 128, 511, 1023, 1500, 2047, 3070, R - 2, R - 1], np.int32)
    ref = oracle.synthesis_sep(alm_in.astype(np.complex128), NS2, L2, L2, rings)
    g = oracle.ring_geometry(NS2)
    got = np.concatenate([smap[:, g["start"][y]: g["start"][y] + g["nphi"][y]] for y in rings], axis=1)
    assert rel_err(got, ref) <= 1e-5
    ms = [0, 1, 2, 127, 128, 1024, 2047, 3000, 3071]
    ls, mm = [], []
    r = syn.rng(78)
    for m in ms:
        cand = sorted(set([m, min(m + 1, L2), min(m + 127, L2), min(m + 128, L2), L2]
                          + list(r.integers(m, L2 + 1, 3))))
        ls += cand
        mm += [m] * len(cand)
    ls, mm = np.array(ls, np.int32), np.array(mm, np.int32)
    ref = oracle.analysis_sep(maps.astype(np.float64), L2, ls, mm, weights="equal")
    assert rel_err(a[:, oracle.alm_index(L2, ls, mm)], ref) <= 1e-5


def test_cfg2_tensor_core_adjoints_and_gradients_sampled():
    """Nside 1024, lmax 3071, 8 channels on the benchmark's tensor-core plan
    (FP16 hi/lo): both adjoints (Sec. III-F) and both gradient forms against
    the oracle on sampled coefficients and rings.  Y^dagger p is the analysis
    sum with unit weights; W Y a the synthesis times the ring weight; the
    gradients are D Y^dagger g (Im of m = 0 dropped) and W Y D^-1 g, with
    D = 1 at m = 0 and 2 above (the complex-gradient convention)."""
    maps = syn.white_maps(syn.SEED_BASE + 12, NS2, B2).astype(np.float32)
    alm_in = syn.gaussian_alm(syn.SEED_BASE + 13, L2, L2, B2, power=2.0).astype(np.complex64)
    h = hpx()
    dm, da = torch.from_numpy(maps).cuda(), torch.from_numpy(alm_in).cuda()
    with h.Plan(NS2, L2, L2, B2, "f32", lambda_table=True, tensor_cores=True) as pc:
        adj_a = pc.alm2map_adjoint(dm).cpu().numpy()
        grad_a = pc.alm2map_grad(dm).cpu().numpy()
        adj_m = pc.map2alm_adjoint(da).cpu().numpy()
        grad_m = pc.map2alm_grad(da).cpu().numpy()
        pc.device_status()
    ms = [0, 1, 2, 127, 128, 1024, 2047, 3000, 3071]
    ls, mm = [], []
    r = syn.rng(79)
    for m in ms:
        cand = sorted(set([m, min(m + 1, L2), min(m + 127, L2), min(m + 128, L2), L2]
                          + list(r.integers(m, L2 + 1, 3))))
        ls += cand
        mm += [m] * len(cand)
    ls, mm = np.array(ls, np.int32), np.array(mm, np.int32)
    idx = oracle.alm_index(L2, ls, mm)
    ref = oracle.analysis_sep(maps.astype(np.float64), L2, ls, mm, weights=None)
    assert rel_err(adj_a[:, idx], ref) <= 1e-5
    Dm = np.where(mm == 0, 1.0, 2.0)
    gref = Dm * ref
    gref[:, mm == 0] = gref[:, mm == 0].real
    assert rel_err(grad_a[:, idx], gref) <= 1e-5
    R = 4 * NS2 - 1
    rings = np.array([0, 1, 2, 127, 128, 511, 1023, 1500, 2047, 3070, R - 2, R - 1], np.int32)
    g = oracle.ring_geometry(NS2)

    def pick(x):
        return np.concatenate([x[:, g["start"][y]: g["start"][y] + g["nphi"][y]] for y in rings], axis=1)
    a64 = alm_in.astype(np.complex128)
    ref = oracle.synthesis_sep(a64, NS2, L2, L2, rings, scale="equal")
    assert rel_err(pick(adj_m), ref) <= 1e-5
    _, mall = oracle.lm_arrays(L2, L2)
    ref = oracle.synthesis_sep(a64 / np.where(mall == 0, 1.0, 2.0), NS2, L2, L2, rings, scale="equal")
    assert rel_err(pick(grad_m), ref) <= 1e-5


@pytest.mark.parametrize("kw", [dict(lambda_table=True, tensor_cores=True), dict(lambda_table=True, tensor_cores=True,
                                                                              tf32x3=True), {}],
                         ids=["fp16-split", "tf32x3", "cuda-cores"])
def test_analysis_and_synthesis_on_two_streams(kw):
    """One analysis and one synthesis of a plan running at the same time on
    two streams (their workspaces are apart) give the results of the same
    calls in sequence, bit for bit."""
    nside, lmax, nb = 64, 191, 8
    maps = torch.from_numpy(syn.white_maps(95, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(96, lmax, lmax, nb).astype(np.complex64)).cuda()
    with hpx().Plan(nside, lmax, lmax, nb, "f32", **kw) as p:
        ra, rm = p.map2alm(maps).clone(), p.alm2map(alm).clone()
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        main = torch.cuda.current_stream()
        oa, om = p.empty_alm(), p.empty_map()
        for _ in range(3):
            sa.wait_stream(main)
            sb.wait_stream(main)
            p.map2alm(maps, out=oa, stream=sa)
            p.alm2map(alm, out=om, stream=sb)
            main.wait_stream(sa)
            main.wait_stream(sb)
            torch.cuda.synchronize()
            assert torch.equal(oa, ra) and torch.equal(om, rm)
        p.device_status()


@pytest.mark.parametrize("kw", [dict(lambda_table=True, tensor_cores=True), {}], ids=["fp16-split", "cuda-cores"])
def test_n_forms_and_their_concurrency(kw):
    """The _n forms (the first n channels of the plan's batch, as the server
    packs them) equal the full calls' first n channels bit for bit (the
    16-bit operand scales are per channel), and an _n analysis and an _n
    synthesis with different n may run at once on two streams."""
    nside, lmax, nb = 64, 191, 8
    maps = torch.from_numpy(syn.white_maps(97, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(98, lmax, lmax, nb).astype(np.complex64)).cuda()
    with hpx().Plan(nside, lmax, lmax, nb, "f32", **kw) as p:
        fa, fm = p.map2alm(maps).clone(), p.alm2map(alm).clone()
        a5, m3 = p.empty_alm(), p.empty_map()
        p.map2alm_n(5, maps, a5)
        p.alm2map_n(3, alm, m3)
        torch.cuda.synchronize()
        assert torch.equal(a5[:5], fa[:5]) and torch.equal(m3[:3], fm[:3])
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        main = torch.cuda.current_stream()
        a8, m4 = p.empty_alm(), p.empty_map()
        for _ in range(3):
            sa.wait_stream(main)
            sb.wait_stream(main)
            p.map2alm_n(8, maps, a8, stream=sa)
            p.alm2map_n(4, alm, m4, stream=sb)
            main.wait_stream(sa)
            main.wait_stream(sb)
            torch.cuda.synchronize()
            assert torch.equal(a8, fa) and torch.equal(m4[:4], fm[:4])
        p.device_status()
