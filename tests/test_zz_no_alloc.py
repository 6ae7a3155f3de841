"""hpx_map2alm_noalloc -- the analysis for callers that must not allocate
device memory when they transform (their memory belongs to another allocator
or pool, or their loop cannot afford the device-wide synchronisation of
cudaMalloc / cudaFree) -- through the C ABI.

Its intermediate spectra live in one fixed device array shared by all calls,
so two calls in a row on different inputs must each match the regular entry
point and the FP64 oracle (the second must not see the first one's data),
and a call after the first must leave the device's free memory and the torch
allocator untouched.  This file is collected last so that a run stopping at
the first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2510_01785_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def rel(a, b):
    """Largest per-channel relative L2 error of a against b ([nbatch][...])."""
    a = torch.as_tensor(a).to(torch.complex128).reshape(a.shape[0], -1)
    b = torch.as_tensor(b).to(torch.complex128).reshape(b.shape[0], -1)
    return float(((a - b).abs().pow(2).sum(1).sqrt() / b.abs().pow(2).sum(1).sqrt()).max())


def call(p, maps, out):
    from paper_2510_01785_gb300._lib import lib
    st = lib().hpx_map2alm_noalloc(p._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib().hpx_last_error()


@pytest.mark.parametrize("dtype,nside,lmax,nbatch", [("f32", 64, 191, 4), ("f64", 32, 95, 3),
                                                     ("f32", 256, 767, 5)])
def test_noalloc_matches_map2alm_twice(dtype, nside, lmax, nbatch):
    import paper_2510_01785_gb300 as hpx
    rdt = torch.float64 if dtype == "f64" else torch.float32
    with hpx.Plan(nside, lmax, lmax, nbatch, dtype) as p:
        for k, seed in enumerate([11, 12]):
            maps = torch.from_numpy(syn.white_maps(seed, nside, nbatch)).to("cuda", rdt)
            ref = p.map2alm(maps)
            out = p.empty_alm()
            call(p, maps, out)
            torch.cuda.synchronize()
            assert rel(out.cpu(), ref.cpu()) <= TOL[dtype], (k, rel(out.cpu(), ref.cpu()))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_the_oracle_twice(dtype):
    """Per channel against the FP64 oracle's analysis, on two different maps
    in a row (band-limited, then white noise), at the FP64 / FP32 bars."""
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 32, 95, 3
    rdt = torch.float64 if dtype == "f64" else torch.float32
    alm = syn.gaussian_alm(syn.SEED_BASE + 71, lmax, lmax, nb, power=2.0)
    inputs = [oracle.alm2map(alm, nside, lmax, lmax), syn.white_maps(syn.SEED_BASE + 72, nside, nb)]
    with hpx.Plan(nside, lmax, lmax, nb, dtype) as p:
        for k, m in enumerate(inputs):
            ref = oracle.map2alm(m, lmax, lmax)
            maps = torch.from_numpy(np.ascontiguousarray(m)).to("cuda", rdt)
            out = p.empty_alm()
            call(p, maps, out)
            torch.cuda.synchronize()
            e = rel(out.cpu(), torch.from_numpy(ref))
            assert e <= TOL[dtype], (k, e)


def test_noalloc_allocates_nothing_after_the_first_call():
    """After a first call (which may load the array's module), further calls
    change neither the device's free memory nor the torch allocator."""
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 64, 191, 4
    with hpx.Plan(nside, lmax, lmax, nb, "f32") as p:
        maps = torch.from_numpy(syn.white_maps(21, nside, nb)).to("cuda", torch.float32)
        out = p.empty_alm()
        call(p, maps, out)
        torch.cuda.synchronize()
        ref = out.clone()
        free0, _ = torch.cuda.mem_get_info()
        alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        for _ in range(3):
            call(p, maps, out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
        assert torch.equal(out, ref)


@pytest.mark.parametrize("tf32x3", [False, True])
def test_noalloc_on_tensor_core_plans(tf32x3):
    """On a tensor-core plan the call runs the CUDA-core analysis: on the
    plan's FP32 table (3xTF32 plans) or recomputing lambda (FP16-split
    plans, whose 16-bit table the CUDA-core kernels cannot read)."""
    import paper_2510_01785_gb300 as hpx
    nside, lmax, nb = 64, 191, 3
    maps = torch.from_numpy(syn.white_maps(13, nside, nb)).to("cuda", torch.float32)
    with hpx.Plan(nside, lmax, lmax, nb, "f32") as pr:
        ref = pr.map2alm(maps)
    with hpx.Plan(nside, lmax, lmax, nb, "f32", lambda_table=True, tensor_cores=True, tf32x3=tf32x3) as p:
        out = p.empty_alm()
        call(p, maps, out)
        torch.cuda.synchronize()
        assert rel(out.cpu(), ref.cpu()) <= TOL["f32"]


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
