"""GPU transforms against the FP64 oracle, element by element, on the same
seeded inputs.

Tolerances (relative L2 per channel, worst channel; Sec. IV-A reports
errors the same way):
  FP64 path  <= 1e-12
  FP32 path  <= 1e-5
Full outputs at sizes the oracle finishes in seconds (several l-blocks,
cluster ranks and ragged channel groups); sampled outputs plus an exact
adjoint identity at Nside 1024, lmax 3071, 8 channels.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def hpx():
    import paper_2510_01785_gb300 as h
    return h


def rel_err(got, ref):
    """max over channels of ||got_b - ref_b|| / ||ref_b||."""
    got = np.atleast_2d(np.asarray(got))
    ref = np.atleast_2d(np.asarray(ref))
    num = np.linalg.norm((got - ref).reshape(ref.shape[0], -1), axis=1)
    den = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def to_dev(x, dtype):
    if np.iscomplexobj(x):
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if dtype == "f64" else np.complex64)))
    else:
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if dtype == "f64" else np.float32)))
    return t.cuda()


def rounded(x, dtype):
    """The input exactly as the GPU sees it, widened back to float64."""
    if dtype == "f64":
        return x
    if np.iscomplexobj(x):
        return x.astype(np.complex64).astype(np.complex128)
    return x.astype(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nside", [1, 2, 8, 64, 1024])
def test_ring_table_matches_oracle(nside):
    p = hpx().Plan(nside, 3, 3, 1, "f64")
    got = p.ring_table()
    ref = oracle.ring_geometry(nside)
    for k in ["start", "nphi", "sigma"]:
        assert np.array_equal(got[k], ref[k]), k
    for k in ["z", "sinth"]:
        assert np.all(np.abs(got[k] - ref[k]) <= np.spacing(np.abs(ref[k]) + 1e-300)), k
    p.close()


# --------------------------------------------------------------------------
# full-output parity at small sizes
# --------------------------------------------------------------------------
CASES = [
    # nside, lmax, mmax, nbatch
    (1, 2, 2, 1),
    (2, 5, 5, 3),
    (4, 11, 11, 2),
    (8, 23, 23, 5),       # Bluestein rings (i = 3, 5, 6, 7)
    (8, 40, 30, 2),       # lmax > 3 nside - 1: every ring aliases
    (16, 47, 20, 3),      # mmax < lmax
    (32, 0, 0, 1),        # lmax = 0
    (32, 95, 95, 17),     # 17 channels: two channel groups, ragged
    (64, 191, 191, 3),    # 128 ring pairs, 6 l-blocks
    (128, 383, 383, 2),   # 256 pairs: one full CTA per cluster
    (256, 400, 380, 1),   # 512 pairs: cluster of 2, partial top block
]


@pytest.fixture(scope="module")
def small_refs():
    cache = {}

    def get(case):
        if case not in cache:
            nside, lmax, mmax, nb = case
            maps = syn.white_maps(syn.SEED_BASE + 100 + nside, nside, nb)
            alm = syn.gaussian_alm(syn.SEED_BASE + 200 + nside, lmax, mmax, nb, power=1.0)
            out = {}
            for dt in ["f64", "f32"]:
                m, a = rounded(maps, dt), rounded(alm, dt)
                out[dt] = dict(
                    maps=m, alm=a,
                    map2alm=oracle.map2alm(m, lmax, mmax),
                    alm2map=oracle.alm2map(a, nside, lmax, mmax),
                    map2alm_adjoint=oracle.map2alm_adjoint(a, nside, lmax, mmax),
                    alm2map_adjoint=oracle.alm2map_adjoint(m, lmax, mmax))
            cache[case] = out
        return cache[case]
    return get


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=[f"ns{c[0]}-l{c[1]}-m{c[2]}-b{c[3]}" for c in CASES])
def test_full_parity(case, dtype, small_refs):
    nside, lmax, mmax, nb = case
    ref = small_refs(case)[dtype]
    with hpx().Plan(nside, lmax, mmax, nb, dtype) as p:
        maps = to_dev(ref["maps"], dtype)
        alm = to_dev(ref["alm"], dtype)
        got = {
            "map2alm": p.map2alm(maps),
            "alm2map": p.alm2map(alm),
            "map2alm_adjoint": p.map2alm_adjoint(alm),
            "alm2map_adjoint": p.alm2map_adjoint(maps),
        }
        torch.cuda.synchronize()
        for k, v in got.items():
            e = rel_err(v.cpu().numpy(), ref[k])
            assert e <= TOL[dtype], (k, e)
        # real input: Im a_l0 is exactly zero
        a = got["map2alm"].cpu().numpy()
        assert np.all(a[:, : lmax + 1].imag == 0.0)


def test_cfg1_fp64_round_trip():
    """Nside 32, lmax = mmax = 95, one channel, FP64: the map is the oracle's
    synthesis of seeded a_lm ~ N(0, (l+1)^-2); map2alm and alm2map both match
    the oracle to 1e-12."""
    nside, lmax = 32, 95
    alm = syn.gaussian_alm(syn.SEED_BASE + 1, lmax, lmax, 1, power=2.0)
    maps = oracle.alm2map(alm, nside, lmax, lmax)
    ref_alm = oracle.map2alm(maps, lmax, lmax)
    with hpx().Plan(nside, lmax, lmax, 1, "f64") as p:
        got_map = p.alm2map(to_dev(alm, "f64")).cpu().numpy()
        got_alm = p.map2alm(to_dev(maps, "f64")).cpu().numpy()
    assert rel_err(got_map, maps) <= 1e-12
    assert rel_err(got_alm, ref_alm) <= 1e-12


# --------------------------------------------------------------------------
# Nside 1024, lmax 3071, 8 channels (the benchmark's configuration)
# --------------------------------------------------------------------------
NS2, L2, B2 = 1024, 3071, 8


@pytest.fixture(scope="module")
def big():
    maps = syn.white_maps(syn.SEED_BASE + 2, NS2, B2).astype(np.float32)
    alm = syn.gaussian_alm(syn.SEED_BASE + 3, L2, L2, B2, power=2.0).astype(np.complex64)
    p = hpx().Plan(NS2, L2, L2, B2, "f32")
    dmaps, dalm = to_dev(maps, "f32"), to_dev(alm, "f32")
    out = dict(maps=maps, alm=alm, plan=p, dmaps=dmaps, dalm=dalm,
               a=p.map2alm(dmaps), s=p.alm2map(dalm))
    torch.cuda.synchronize()
    yield out
    p.close()


def test_cfg2_map2alm_sampled(big):
    ms = [0, 1, 2, 3, 511, 1024, 2047, 2048, 3070, 3071]
    ls, mm = [], []
    r = syn.rng(77)
    for m in ms:
        cand = sorted(set([m, min(m + 1, L2), L2] + list(r.integers(m, L2 + 1, 3))))
        ls += cand
        mm += [m] * len(cand)
    ls, mm = np.array(ls, np.int32), np.array(mm, np.int32)
    ref = oracle.analysis_sep(big["maps"].astype(np.float64), L2, ls, mm, weights="equal")
    got = big["a"].cpu().numpy()[:, oracle.alm_index(L2, ls, mm)]
    assert rel_err(got, ref) <= 1e-5


def test_cfg2_alm2map_sampled(big):
    R = 4 * NS2 - 1
    rings = np.array([0, 1, 2, 511, 1022, 1023, 1500, 2047, 3070, R - 2, R - 1], np.int32)
    ref = oracle.synthesis_sep(big["alm"].astype(np.complex128), NS2, L2, L2, rings)
    g = oracle.ring_geometry(NS2)
    s = big["s"].cpu().numpy()
    got = np.concatenate([s[:, g["start"][y]: g["start"][y] + g["nphi"][y]] for y in rings], axis=1)
    assert rel_err(got, ref) <= 1e-5


def test_cfg2_adjoint_identity(big):
    """<Y a, p> = <a, Y^dagger p>_full holds at any size."""
    p = big["plan"]
    Ya = big["s"].double()
    Ytp = p.alm2map_adjoint(big["dmaps"]).to(torch.complex128)
    pm = big["dmaps"].double()
    a = big["dalm"].to(torch.complex128)
    lhs = (Ya * pm).sum(dim=1)
    w = torch.full((p.nalm,), 2.0, dtype=torch.float64, device=a.device)
    w[: L2 + 1] = 1.0
    rhs = (w * (a.conj() * Ytp).real).sum(dim=1)
    rel = ((lhs - rhs).abs() / (Ya.norm(dim=1) * pm.norm(dim=1))).max().item()
    assert rel < 1e-6


def test_max_size_sampled():
    """The largest plan: Nside 2048, lmax 6143, 4 FP32 channels, lambda
    recomputed (its tables would not fit).  Sampled coefficients at the
    extreme and aliased m (4096 = the belt ring length 8192 / 2) and sampled
    rings at both poles, the last cap ring and the equator, against tier B."""
    ns, lm, nb = 2048, 6143, 4
    maps = syn.white_maps(syn.SEED_BASE + 4, ns, nb).astype(np.float32)
    alm = syn.gaussian_alm(syn.SEED_BASE + 5, lm, lm, nb, power=2.0).astype(np.complex64)
    with hpx().Plan(ns, lm, lm, nb, "f32") as p:
        got_a = p.map2alm(to_dev(maps, "f32")).cpu().numpy()
        got_s = p.alm2map(to_dev(alm, "f32")).cpu().numpy()
    ls, mm = [], []
    r = syn.rng(78)
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


def test_cfg2_deterministic_and_stream(big):
    p = big["plan"]
    s = torch.cuda.Stream()
    out = p.empty_alm()
    with torch.cuda.stream(s):
        p.map2alm(big["dmaps"], out=out)
    s.synchronize()
    assert torch.equal(out, big["a"])


def test_host_entry_points_match_device():
    nside, lmax, nb = 16, 47, 2
    maps = syn.white_maps(5, nside, nb).astype(np.float32)
    alm = syn.gaussian_alm(6, lmax, lmax, nb).astype(np.complex64)
    with hpx().Plan(nside, lmax, lmax, nb, "f32") as p:
        a_host = p.map2alm_host(maps).numpy()
        a_dev = p.map2alm(to_dev(maps, "f32")).cpu().numpy()
        m_host = p.alm2map_host(alm).numpy()
        m_dev = p.alm2map(to_dev(alm, "f32")).cpu().numpy()
    assert np.array_equal(a_host, a_dev)
    assert np.array_equal(m_host, m_dev)


def test_bad_arguments_raise():
    h = hpx()
    with h.Plan(8, 10, 10, 2, "f32") as p:
        with pytest.raises(ValueError):
            p.map2alm(torch.zeros((1, p.npix), device="cuda"))
        with pytest.raises(ValueError):
            p.alm2map(torch.zeros((2, p.nalm), device="cuda", dtype=torch.complex128))
    with pytest.raises(RuntimeError):
        h.Plan(12, 10, 10, 1, "f32")


# --------------------------------------------------------------------------
# plan-resident lambda table: same recurrence values, so identical results
# --------------------------------------------------------------------------
TABLE_CASES = [(1, 2, 2, 1), (2, 5, 5, 3), (8, 40, 30, 2), (16, 47, 20, 3), (64, 191, 191, 3),
               (256, 400, 380, 1), (512, 1535, 1535, 2)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", TABLE_CASES, ids=[f"ns{c[0]}-l{c[1]}-m{c[2]}-b{c[3]}" for c in TABLE_CASES])
def test_table_mode_equals_recompute(case, dtype):
    nside, lmax, mmax, nb = case
    maps = to_dev(syn.white_maps(31, nside, nb), dtype)
    alm = to_dev(syn.gaussian_alm(32, lmax, mmax, nb, power=1.0), dtype)
    h = hpx()
    with h.Plan(nside, lmax, mmax, nb, dtype) as pr, h.Plan(nside, lmax, mmax, nb, dtype, lambda_table=True) as pt:
        assert pt.device_bytes > pr.device_bytes
        for op, x in (("map2alm", maps), ("alm2map", alm), ("map2alm_adjoint", alm), ("alm2map_adjoint", maps)):
            a = getattr(pr, op)(x)
            b = getattr(pt, op)(x)
            torch.cuda.synchronize()
            assert torch.equal(a, b), op


def test_cfg2_table_mode_equals_recompute(big):
    h = hpx()
    with h.Plan(NS2, L2, L2, B2, "f32", lambda_table=True) as pt:
        assert torch.equal(pt.map2alm(big["dmaps"]), big["a"])
        assert torch.equal(pt.alm2map(big["dalm"]), big["s"])


def test_plans_of_different_sizes_interleaved():
    """A plan keeps working after a smaller one is created (per-function
    launch limits are global and must not shrink under a live plan)."""
    h = hpx()
    big_p = h.Plan(64, 191, 191, 2, "f32")
    x = to_dev(syn.white_maps(71, 64, 2), "f32")
    ref = big_p.map2alm(x).clone()
    small = h.Plan(4, 11, 11, 1, "f32")
    small.map2alm(to_dev(syn.white_maps(72, 4, 1), "f32"))
    again = big_p.map2alm(x)
    m = big_p.alm2map(ref)
    torch.cuda.synchronize()
    assert torch.equal(again, ref) and torch.isfinite(m).all()
    small.close()
    big_p.close()
