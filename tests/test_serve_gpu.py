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
