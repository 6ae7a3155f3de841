"""hpx_map2alm_noalloc -- the analysis for callers that must not allocate
device memory when they transform -- against hpx_map2alm, through the C ABI.

Its intermediate spectra live in one fixed device array shared by all calls,
so two calls in a row on different inputs must each match the regular entry
point (the second must not see the first one's data).  This file is collected
last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dtype,nside,lmax,nbatch", [("f32", 64, 191, 4), ("f64", 32, 95, 3),
                                                     ("f32", 256, 767, 5)])
def test_noalloc_matches_map2alm_twice(dtype, nside, lmax, nbatch):
    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300._lib import lib
    rdt = torch.float64 if dtype == "f64" else torch.float32
    with hpx.Plan(nside, lmax, lmax, nbatch, dtype) as p:
        stream = torch.cuda.current_stream().cuda_stream
        for call, seed in enumerate([11, 12]):
            maps = torch.from_numpy(syn.white_maps(seed, nside, nbatch)).to("cuda", rdt)
            ref = p.map2alm(maps)
            out = p.empty_alm()
            st = lib().hpx_map2alm_noalloc(p._h, ctypes.c_void_p(maps.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
            assert st == 0, lib().hpx_last_error()
            torch.cuda.synchronize()
            assert rel(out, ref) <= TOL[dtype], (call, rel(out, ref))


@pytest.mark.parametrize("tf32x3", [False, True])
def test_noalloc_on_tensor_core_plans(tf32x3):
    """On a tensor-core plan the call runs the CUDA-core analysis: on the
    plan's FP32 table (3xTF32 plans) or recomputing lambda (FP16-split
    plans, whose 16-bit table the CUDA-core kernels cannot read)."""
    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300._lib import lib
    nside, lmax, nb = 64, 191, 3
    maps = torch.from_numpy(syn.white_maps(13, nside, nb)).to("cuda", torch.float32)
    with hpx.Plan(nside, lmax, lmax, nb, "f32") as pr:
        ref = pr.map2alm(maps)
    with hpx.Plan(nside, lmax, lmax, nb, "f32", lambda_table=True, tensor_cores=True, tf32x3=tf32x3) as p:
        out = p.empty_alm()
        st = lib().hpx_map2alm_noalloc(p._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, lib().hpx_last_error()
        torch.cuda.synchronize()
        assert rel(out, ref) <= TOL["f32"]


def test_noalloc_rejects_plans_beyond_its_array():
    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300._lib import lib
    with hpx.Plan(512, 16, 16, 2, "f32") as p:  # 2 x 1.57e6 bins x 8 B > 16 MiB
        maps = torch.zeros((2, p.npix), device="cuda")
        out = p.empty_alm()
        st = lib().hpx_map2alm_noalloc(p._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       None)
        assert st == 1
        assert b"16777216" in lib().hpx_last_error()
