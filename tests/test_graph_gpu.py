"""Stream capture: the device-buffer transforms of a resident plan allocate
nothing and never wait on the host, so a CUDA graph can record them; its
replays give the eager calls' results bit for bit.  From Nside 512 the ring
stages fork onto the plan's second stream and join back, which the capture
records too."""
import numpy as np
import pytest
import torch

from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [(32, 95, 1, "f64", {}), (64, 191, 8, "f32", {}),
                                  (64, 191, 8, "f32", dict(lambda_table=True, tensor_cores=True)),
                                  (64, 191, 9, "bf16x3", {}), (512, 127, 2, "f32", {})],
                         ids=["f64", "f32-recompute", "f32-tensor-cores", "bf16x3",
                              "f32-nside512-forked-ring-stages"])
def test_transforms_replay_from_a_cuda_graph(case):
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb, dtype, kw = case
    rdt = torch.float64 if dtype == "f64" else torch.float32
    with hpx.Plan(nside, lmax, lmax, nb, dtype, **kw) as p:
        maps = torch.from_numpy(syn.white_maps(70 + nb, nside, nb)).to("cuda", rdt)
        alm = p.map2alm(maps).clone()
        refs = [p.map2alm(maps).clone(), p.alm2map(alm).clone(), p.alm2map_adjoint(maps).clone(),
                p.map2alm_adjoint(alm).clone()]
        outs = [p.empty_alm(), p.empty_map(), p.empty_alm(), p.empty_map()]

        def calls():
            p.map2alm(maps, out=outs[0])
            p.alm2map(alm, out=outs[1])
            p.alm2map_adjoint(maps, out=outs[2])
            p.map2alm_adjoint(alm, out=outs[3])
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            calls()  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            calls()
        for _ in range(2):
            for o in outs:
                o.zero_()
            g.replay()
            torch.cuda.synchronize()
            for o, r in zip(outs, refs):
                assert torch.equal(o, r)
        p.device_status()
