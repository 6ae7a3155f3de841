"""Pipelined host-buffer entry points: queued calls with alternating I/O
slots give exactly the blocking calls' results, for interleaved analyses
and syntheses."""
import numpy as np
import pytest
import torch

from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [{}, dict(lambda_table=True, tensor_cores=True)])
def test_pipelined_host_calls_match_blocking(kw):
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 64, 191, 3
    with hpx.Plan(nside, lmax, lmax, nb, "f32", **kw) as p:
        maps = [torch.from_numpy(syn.white_maps(900 + i, nside, nb).astype(np.float32)).pin_memory()
                for i in range(3)]
        alms = [torch.from_numpy(syn.gaussian_alm(910 + i, lmax, lmax, nb).astype(np.complex64)).pin_memory()
                for i in range(3)]
        ref_a = [p.map2alm_host(m).clone() for m in maps]
        ref_m = [p.alm2map_host(a).clone() for a in alms]
        out_a = [torch.empty_like(r).pin_memory() for r in ref_a]
        out_m = [torch.empty_like(r).pin_memory() for r in ref_m]
        for i in range(3):
            p.map2alm_host_async(maps[i], out_a[i])
            p.alm2map_host_async(alms[i], out_m[i])
        p.host_sync()
        for i in range(3):
            assert torch.equal(out_a[i], ref_a[i]) and torch.equal(out_m[i], ref_m[i]), i
