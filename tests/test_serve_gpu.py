"""The continuously batching server on the GPU: every request's result is
the same served alone and in the mix (batched with other requests, slots of
several geometries running concurrently on their own streams)."""
import numpy as np
import pytest
import torch

from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_results_alone_equal_results_in_the_mix():
    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300.serve import GpuExecutor, Server, latency_report, make_requests

    reqs = make_requests(11, rate=4000.0, duration=0.02, nside_weights={8: 1, 16: 1, 32: 1, 64: 1},
                         max_channels=8)
    assert len(reqs) >= 40
    for r in reqs:
        if r.op == "map2alm":
            r.x = torch.from_numpy(syn.white_maps(1000 + r.rid, r.nside, r.nch).astype(np.float32)).cuda()
        else:
            r.x = torch.from_numpy(syn.gaussian_alm(2000 + r.rid, r.lmax, r.lmax, r.nch).astype(np.complex64)).cuda()
    torch.cuda.synchronize()
    srv = Server(GpuExecutor(), hbm_cap_bytes=4e9, max_channels=16, max_slots_per_key=2)
    srv.run(reqs, drain_s=60.0)
    torch.cuda.synchronize()
    rep = latency_report(reqs)
    assert rep["served"] == len(reqs) and rep["errors"] == 0
    assert srv.batches < len(reqs)  # requests were batched together
    for r in reqs:
        with hpx.Plan(r.nside, r.lmax, r.lmax, r.nch, "f32") as p:
            alone = p.map2alm(r.x) if r.op == "map2alm" else p.alm2map(r.x)
            torch.cuda.synchronize()
        err = (r.y - alone).abs().max().item() / max(alone.abs().max().item(), 1e-30)
        assert err <= 1e-6, (r.rid, r.op, r.nside, r.nch, err)


def _rel(got, ref):
    got, ref = np.atleast_2d(got), np.atleast_2d(ref)
    num = np.linalg.norm((got - ref).reshape(ref.shape[0], -1), axis=1)
    return float(np.max(num / np.maximum(np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1), 1e-300)))


@pytest.mark.parametrize("tables,streamed", [((32, 128), ()), ((16,), (64, 256))], ids=["tables", "streamed"])
def test_served_results_match_the_oracle_with_tables_and_eviction(tables, streamed):
    """Every served result against the FP64 oracle (relative L2 per channel
    <= 1e-5, the FP32 bar): geometries up to Nside 256, tensor-core table
    slots beside CUDA-core recomputing ones, or streamed-lambda tensor-core
    slots (lambda recomputed per batch into staging blocks) beside a table
    slot, batches wider than one request, and an HBM cap small enough that
    idle slots are evicted."""
    import oracle
    from paper_2510_01785_gb300.serve import GpuExecutor, Server, latency_report, make_requests

    weights = {16: 1, 32: 1, 64: 1, 128: 1, 256: 1}
    reqs = make_requests(23, rate=3000.0, duration=0.012, nside_weights=weights, max_channels=6)
    assert len(reqs) >= 20
    for r in reqs:
        if r.op == "map2alm":
            alm = syn.gaussian_alm(3000 + r.rid, r.lmax, r.lmax, r.nch, power=2.0)
            r.x_np = oracle.alm2map(alm, r.nside, r.lmax, r.lmax) if r.nside <= 64 else \
                syn.white_maps(3000 + r.rid, r.nside, r.nch)
            r.x = torch.from_numpy(r.x_np.astype(np.float32)).cuda()
        else:
            r.x_np = syn.gaussian_alm(4000 + r.rid, r.lmax, r.lmax, r.nch).astype(np.complex64)
            r.x = torch.from_numpy(r.x_np).cuda()
    ex = GpuExecutor(lambda_table_nsides=tables, batch_channels={ns: 12 for ns in weights}, streamed_nsides=streamed)
    sizes = sorted(ex.slot_bytes(ns, 3 * ns - 1, 12) for ns in weights)
    cap = sizes[-1] + 1  # any one slot fits, not all five geometries
    srv = Server(ex, hbm_cap_bytes=cap, max_channels=6, max_slots_per_key=1)
    srv.run(reqs, drain_s=120.0)
    torch.cuda.synchronize()
    rep = latency_report(reqs)
    assert rep["served"] == len(reqs) and rep["errors"] == 0
    assert srv.batches < len(reqs) and srv.evictions > 0 and srv.peak_bytes <= cap
    for r in reqs:
        y = r.y.cpu().numpy()
        x = r.x_np.astype(np.float64) if r.op == "map2alm" else r.x_np.astype(np.complex128)
        if r.nside <= 128:
            ref = oracle.map2alm(x, r.lmax, r.lmax) if r.op == "map2alm" else \
                oracle.alm2map(x, r.nside, r.lmax, r.lmax)
            got = y
        elif r.op == "map2alm":  # sampled coefficients, including l = m, lmax and m = lmax
            g = syn.rng(r.rid)
            ms = np.array([0, 1, r.lmax // 2, r.lmax - 1, r.lmax], np.int32)
            ls = np.array([min(m + int(k), r.lmax) for m in ms for k in (0, 1, g.integers(0, r.lmax + 1))], np.int32)
            ms = np.repeat(ms, 3)
            ls = np.maximum(ls, ms)
            ref = oracle.analysis_sep(x, r.lmax, ls, ms, weights="equal")
            got = y[:, oracle.alm_index(r.lmax, ls, ms)]
        else:  # sampled rings: both poles, a cap ring, the equator
            R = 4 * r.nside - 1
            rings = np.array([0, 1, r.nside - 1, 2 * r.nside - 1, R - 1], np.int32)
            ref = oracle.synthesis_sep(x, r.nside, r.lmax, r.lmax, rings)
            geo = oracle.ring_geometry(r.nside)
            got = np.concatenate([y[:, geo["start"][k]: geo["start"][k] + geo["nphi"][k]] for k in rings], axis=1)
        e = _rel(got, ref)
        assert e <= 1e-5, (r.rid, r.op, r.nside, r.nch, e)
