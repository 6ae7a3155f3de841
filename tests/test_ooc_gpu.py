"""Out-of-core lambda tables (Sec. III-G): pinned host tables streamed per
block of m through two staging buffers give the resident plan's results bit
for bit (same tables, same tile kernels, launched per block)."""
import numpy as np
import pytest
import torch

from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "fp16", "bf16x3"])
@pytest.mark.parametrize("case", [(64, 191, 191, 3), (128, 383, 300, 9)])
def test_out_of_core_equals_resident(case, dtype):
    import paper_2510_01785_gb300 as hpx
    nside, lmax, mmax, nb = case
    maps = torch.from_numpy(syn.white_maps(800 + nside, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(801 + nside, lmax, mmax, nb).astype(np.complex64)).cuda()
    kw = dict(lambda_table=True, tensor_cores=True) if dtype == "f32" else {}
    with hpx.Plan(nside, lmax, mmax, nb, dtype, **kw) as pr, \
            hpx.Plan(nside, lmax, mmax, nb, dtype, out_of_core=True, stage_bytes=1 << 20) as po:
        assert po.host_bytes == pr.table_bytes + pr.column_table_bytes
        assert po.table_bytes == pr.table_bytes and po.device_bytes < pr.device_bytes
        for op, x in (("map2alm", maps), ("alm2map", alm), ("alm2map_adjoint", maps), ("map2alm_adjoint", alm)):
            a = getattr(pr, op)(x)
            for _ in range(2):  # the staging buffers alternate across calls
                b = getattr(po, op)(x)
                torch.cuda.synchronize()
                assert torch.equal(a, b), op
        po.device_status()


def test_out_of_core_stage_too_small():
    import paper_2510_01785_gb300 as hpx
    with pytest.raises(RuntimeError):
        hpx.Plan(64, 191, 191, 1, "f32", out_of_core=True, stage_bytes=4096)


def test_out_of_core_needs_the_tensor_core_path():
    import paper_2510_01785_gb300 as hpx
    with pytest.raises(RuntimeError):
        hpx.Plan(16, 47, 47, 1, "f64", out_of_core=True)
