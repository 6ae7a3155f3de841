"""The bounded waits of the tensor-core tile kernels, made to run out on
purpose without a fault: with copies withheld (hpx_plan_test_withhold_copies)
each CTA's first wait for a copy expires after its 1 s limit, with nothing
in flight; the transform must report HPX_ERR_TIMEOUT through the plan's
status word, and the plan must work normally (same bits) once the copies
flow again.  Tiny plans, so every CTA is resident at once and a withheld
transform lasts about a second."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

KINDS = {"fp16-split": ("f32", dict(lambda_table=True, tensor_cores=True)),
         "tf32x3": ("f32", dict(lambda_table=True, tensor_cores=True, tf32x3=True)),
         "bf16": ("bf16", {})}


@pytest.mark.parametrize("kind", list(KINDS))
def test_withheld_copies_time_out_and_the_plan_recovers(kind):
    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300._lib import HpxError, lib
    dtype, kw = KINDS[kind]
    nside, lmax, nb = 2, 5, 2
    maps = torch.from_numpy(syn.white_maps(syn.SEED_BASE + 300, nside, nb).astype(np.float32)).cuda()
    alm = torch.from_numpy(syn.gaussian_alm(syn.SEED_BASE + 301, lmax, lmax, nb).astype(np.complex64)).cuda()
    with hpx.Plan(nside, lmax, lmax, nb, dtype, **kw) as p:
        ref_a, ref_m = p.map2alm(maps).clone(), p.alm2map(alm).clone()
        p.device_status()
        for call in (lambda: p.map2alm(maps), lambda: p.alm2map(alm)):
            assert lib().hpx_plan_test_withhold_copies(p._h, 1) == 0
            call()
            with pytest.raises(HpxError) as err:
                p.device_status()
            assert err.value.status == 4  # HPX_ERR_TIMEOUT
            assert lib().hpx_plan_test_withhold_copies(p._h, 0) == 0
            p.device_status()  # the record was cleared
        assert torch.equal(p.map2alm(maps), ref_a) and torch.equal(p.alm2map(alm), ref_m)
        p.device_status()
    assert lib().hpx_plan_test_withhold_copies(ctypes.c_void_p(), 1) == 1  # null plan
