"""Spherical harmonic transforms on RING-ordered HEALPix grids for NVIDIA GB300.

Python face of libhpx (C ABI in ``include/hpx.h``; method of arXiv 2510.01785,
cuHPX).  Tensors are PyTorch CUDA tensors; this module only checks shapes and
passes ``data_ptr()`` and the current CUDA stream to the library, whose
kernels do all of the work.

* ``Plan``                    -- one (nside, lmax, mmax, nbatch, dtype) setup
* ``Plan.map2alm``            -- a = Y^dagger W p          (Eq. 26-27)
* ``Plan.alm2map``            -- p = Y a                   (Eq. 24-25)
* ``Plan.map2alm_adjoint``    -- W Y a   (adjoint of analysis, Sec. III-F)
* ``Plan.alm2map_adjoint``    -- Y^dagger p (adjoint of synthesis, Sec. III-F)

Maps are real ``[nbatch, 12 nside^2]`` in RING order; coefficients are complex
``[nbatch, nalm]`` packed m-major (index m (2 lmax + 1 - m)/2 + l, m >= 0).
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

__all__ = ["Plan", "nalm", "get_plan", "DTYPES", "reorder", "layout_index", "LAYOUTS"]

DTYPES = {
    "f64": _lib.HPX_F64,
    "f32": _lib.HPX_F32,
    "bf16": _lib.HPX_F32_BF16,
    "bf16x3": _lib.HPX_F32_BF16X3,
    "fp16": _lib.HPX_F32_FP16,
    "fp16x3": _lib.HPX_F32_FP16X3,
}


def nalm(lmax: int, mmax: int | None = None) -> int:
    return int(lib().hpx_nalm(lmax, lmax if mmax is None else mmax))


def _stream_handle(stream, device) -> int:
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Plan:
    """A transform setup: ring geometry, recurrence tables and workspace on
    one GPU.  One analysis and one synthesis may run at once on two streams;
    otherwise one plan serves one call at a time (its workspace); use one
    plan per concurrently used stream."""

    def __init__(self, nside: int, lmax: int, mmax: int | None = None, nbatch: int = 1,
                 dtype: str = "f32", lambda_table: bool = False, device=None,
                 tensor_cores: bool = False, out_of_core: bool = False, stage_bytes: int = 0,
                 tf32x3: bool = False, streamed: bool = False):
        mmax = lmax if mmax is None else mmax
        if dtype not in DTYPES:
            raise ValueError(f"dtype must be one of {sorted(DTYPES)}")
        self.nside, self.lmax, self.mmax, self.nbatch = nside, lmax, mmax, nbatch
        self.dtype = dtype
        self.real_dtype = torch.float64 if dtype == "f64" else torch.float32
        self.complex_dtype = torch.complex128 if dtype == "f64" else torch.complex64
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        self.npix = 12 * nside * nside
        self.nalm = nalm(lmax, mmax)
        self._h = None
        self.lambda_table, self.tensor_cores = lambda_table, tensor_cores
        flags = _lib.HPX_PLAN_LAMBDA_TABLE if lambda_table else _lib.HPX_PLAN_LAMBDA_RECOMPUTE
        if tensor_cores:
            flags |= _lib.HPX_PLAN_TENSOR_CORES
        if tf32x3:  # 3xTF32 split products instead of FP16 hi/lo
            flags |= _lib.HPX_PLAN_TC_TF32X3
        self.tf32x3 = tf32x3
        self.out_of_core, self.streamed = out_of_core, streamed
        if out_of_core and streamed:
            raise ValueError("out_of_core and streamed exclude each other")
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if streamed:  # lambda recomputed per transform into staging slabs, tensor-core products
                check(lib().hpx_plan_create_stream(nside, lmax, mmax, nbatch, DTYPES[dtype],
                                                   _lib.HPX_PLAN_TC_TF32X3 if tf32x3 else 0, int(stage_bytes),
                                                   ctypes.byref(h)), "hpx_plan_create_stream")
            elif out_of_core:
                check(lib().hpx_plan_create_ooc(nside, lmax, mmax, nbatch, DTYPES[dtype], int(stage_bytes),
                                                ctypes.byref(h)), "hpx_plan_create_ooc")
            else:
                check(lib().hpx_plan_create_ex(nside, lmax, mmax, nbatch, DTYPES[dtype], flags,
                                               ctypes.byref(h)), "hpx_plan_create_ex")
        self._h = h

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if self._h is not None and self._h.value:
            lib().hpx_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def device_bytes(self) -> int:
        return int(lib().hpx_plan_device_bytes(self._h))

    def set_ring_weights(self, w) -> None:
        """Per-ring quadrature weights (4 nside - 1 values, north to south) for
        the weighted operators; see weights.ring_weights for a computed set."""
        w = np.ascontiguousarray(np.asarray(w, np.float64))
        check(lib().hpx_plan_set_ring_weights(self._h, ctypes.c_void_p(w.ctypes.data), int(w.size)),
              "hpx_plan_set_ring_weights")

    def device_status(self) -> None:
        """Synchronise and raise HpxError(HPX_ERR_TIMEOUT) if a bounded
        device-side wait of this plan's kernels expired since the last check."""
        check(lib().hpx_plan_device_status(self._h), "hpx_plan_device_status")

    @property
    def table_bytes(self) -> int:
        """Bytes of the plan-resident lambda table (0 when recomputing)."""
        return int(lib().hpx_plan_table_bytes(self._h))

    @property
    def host_bytes(self) -> int:
        """Pinned host bytes of an out-of-core plan's tables (0 otherwise)."""
        return int(lib().hpx_plan_host_bytes(self._h))

    @property
    def column_table_bytes(self) -> int:
        """Bytes of the table copy the tensor-core synthesis reads (0 without it)."""
        return int(lib().hpx_plan_column_table_bytes(self._h))

    # -- argument checks ----------------------------------------------------
    def _map(self, t: torch.Tensor, name: str) -> torch.Tensor:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == self.device):
            raise ValueError(f"{name} must be a CUDA tensor on {self.device}")
        if t.dtype != self.real_dtype or tuple(t.shape) != (self.nbatch, self.npix):
            raise ValueError(f"{name} must be {self.real_dtype} of shape {(self.nbatch, self.npix)}, "
                             f"got {t.dtype} {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _alm(self, t: torch.Tensor, name: str) -> torch.Tensor:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == self.device):
            raise ValueError(f"{name} must be a CUDA tensor on {self.device}")
        if t.dtype != self.complex_dtype or tuple(t.shape) != (self.nbatch, self.nalm):
            raise ValueError(f"{name} must be {self.complex_dtype} of shape {(self.nbatch, self.nalm)}, "
                             f"got {t.dtype} {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def empty_map(self) -> torch.Tensor:
        return torch.empty((self.nbatch, self.npix), dtype=self.real_dtype, device=self.device)

    def empty_alm(self) -> torch.Tensor:
        return torch.empty((self.nbatch, self.nalm), dtype=self.complex_dtype, device=self.device)

    # -- transforms ---------------------------------------------------------
    def _call(self, fn, name, src, dst, stream):
        check(fn(self._h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                 ctypes.c_void_p(_stream_handle(stream, self.device))), name)
        return dst

    def map2alm(self, maps: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """a = Y^dagger W p with w = 4 pi / Npix (Eq. 26-27)."""
        src = self._map(maps, "maps")
        dst = self._alm(out, "out") if out is not None else self.empty_alm()
        return self._call(lib().hpx_map2alm, "hpx_map2alm", src, dst, stream)

    def alm2map(self, alm: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """p = Y a (Eq. 24-25)."""
        src = self._alm(alm, "alm")
        dst = self._map(out, "out") if out is not None else self.empty_map()
        return self._call(lib().hpx_alm2map, "hpx_alm2map", src, dst, stream)

    def map2alm_adjoint(self, alm: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """W Y a: adjoint of map2alm (Sec. III-F)."""
        src = self._alm(alm, "alm")
        dst = self._map(out, "out") if out is not None else self.empty_map()
        return self._call(lib().hpx_map2alm_adjoint, "hpx_map2alm_adjoint", src, dst, stream)

    def alm2map_adjoint(self, maps: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Y^dagger p: adjoint of alm2map (Sec. III-F)."""
        src = self._map(maps, "maps")
        dst = self._alm(out, "out") if out is not None else self.empty_alm()
        return self._call(lib().hpx_alm2map_adjoint, "hpx_alm2map_adjoint", src, dst, stream)

    def _first_n(self, t: torch.Tensor, n: int, cols: int, dtype, name: str) -> torch.Tensor:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == self.device and t.dtype == dtype
                and t.is_contiguous() and t.dim() == 2 and t.shape[0] >= n and t.shape[1] == cols):
            raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor with >= {n} rows of {cols}")
        return t

    def map2alm_n(self, n: int, maps: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """map2alm of the first n (<= nbatch) rows of maps into out."""
        src = self._first_n(maps, n, self.npix, self.real_dtype, "maps")
        dst = self._first_n(out, n, self.nalm, self.complex_dtype, "out")
        check(lib().hpx_map2alm_n(self._h, n, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                  ctypes.c_void_p(_stream_handle(stream, self.device))), "hpx_map2alm_n")
        return dst

    def alm2map_n(self, n: int, alm: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """alm2map of the first n (<= nbatch) rows of alm into out."""
        src = self._first_n(alm, n, self.nalm, self.complex_dtype, "alm")
        dst = self._first_n(out, n, self.npix, self.real_dtype, "out")
        check(lib().hpx_alm2map_n(self._h, n, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                  ctypes.c_void_p(_stream_handle(stream, self.device))), "hpx_alm2map_n")
        return dst

    def map2alm_iter(self, maps: torch.Tensor, niter: int, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        """Analysis with niter steps of iterative refinement (Sec. II-A Eq. 4)."""
        maps = self._map(maps, "maps")
        out = self.empty_alm() if out is None else self._alm(out, "out")
        check(lib().hpx_map2alm_iter(self._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     int(niter), ctypes.c_void_p(_stream_handle(stream, self.device))),
              "hpx_map2alm_iter")
        return out

    def alm2map_grad(self, grad_map: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Backward of alm2map: D Y^dagger g (dL/dRe + i dL/dIm per coefficient)."""
        src = self._map(grad_map, "grad_map")
        dst = self._alm(out, "out") if out is not None else self.empty_alm()
        return self._call(lib().hpx_alm2map_grad, "hpx_alm2map_grad", src, dst, stream)

    def map2alm_grad(self, grad_alm: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Backward of map2alm: W Y D^-1 g."""
        src = self._alm(grad_alm, "grad_alm")
        dst = self._map(out, "out") if out is not None else self.empty_map()
        return self._call(lib().hpx_map2alm_grad, "hpx_map2alm_grad", src, dst, stream)

    # -- host-buffer forms --------------------------------------------------
    def map2alm_host(self, maps: np.ndarray | torch.Tensor, out=None, stream=None):
        """Host map in, host coefficients out (copies inside the call)."""
        src = maps if isinstance(maps, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(maps))
        assert src.device.type == "cpu" and src.dtype == self.real_dtype and src.is_contiguous()
        assert tuple(src.shape) == (self.nbatch, self.npix)
        dst = out if out is not None else torch.empty((self.nbatch, self.nalm), dtype=self.complex_dtype)
        check(lib().hpx_map2alm_host(self._h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                     ctypes.c_void_p(_stream_handle(stream, self.device))), "hpx_map2alm_host")
        return dst

    def map2alm_host_async(self, maps: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """Pipelined host-buffer analysis: queued, complete after host_sync().
        maps and out: pinned CPU tensors kept alive until then."""
        assert maps.is_pinned() and out.is_pinned() and maps.is_contiguous() and out.is_contiguous()
        assert tuple(maps.shape) == (self.nbatch, self.npix) and maps.dtype == self.real_dtype
        assert tuple(out.shape) == (self.nbatch, self.nalm) and out.dtype == self.complex_dtype
        check(lib().hpx_map2alm_host_async(self._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(_stream_handle(stream, self.device))),
              "hpx_map2alm_host_async")
        return out

    def alm2map_host_async(self, alm: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """Pipelined host-buffer synthesis: queued, complete after host_sync()."""
        assert alm.is_pinned() and out.is_pinned() and alm.is_contiguous() and out.is_contiguous()
        assert tuple(alm.shape) == (self.nbatch, self.nalm) and alm.dtype == self.complex_dtype
        assert tuple(out.shape) == (self.nbatch, self.npix) and out.dtype == self.real_dtype
        check(lib().hpx_alm2map_host_async(self._h, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(_stream_handle(stream, self.device))),
              "hpx_alm2map_host_async")
        return out

    def host_sync(self) -> None:
        """Wait for every pipelined host-buffer call."""
        check(lib().hpx_plan_host_sync(self._h), "hpx_plan_host_sync")

    def alm2map_host(self, alm: np.ndarray | torch.Tensor, out=None, stream=None):
        """Host coefficients in, host map out (copies inside the call)."""
        src = alm if isinstance(alm, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(alm))
        assert src.device.type == "cpu" and src.dtype == self.complex_dtype and src.is_contiguous()
        assert tuple(src.shape) == (self.nbatch, self.nalm)
        dst = out if out is not None else torch.empty((self.nbatch, self.npix), dtype=self.real_dtype)
        check(lib().hpx_alm2map_host(self._h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                     ctypes.c_void_p(_stream_handle(stream, self.device))), "hpx_alm2map_host")
        return dst

    # -- measurement support ------------------------------------------------
    STAGES = ("ring_fft_analysis", "legendre_analysis", "legendre_synthesis", "ring_fft_synthesis",
              "analysis_operand_pack", "synthesis_operand_pack")

    def set_timing(self, enable: bool) -> None:
        """Record CUDA events around each stage of every following transform."""
        check(lib().hpx_plan_set_timing(self._h, 1 if enable else 0), "hpx_plan_set_timing")

    def stage_times(self) -> dict:
        """{stage: (total ms, kernel launches)} since the last call; waits."""
        ms = np.zeros(len(self.STAGES), np.float64)
        n = np.zeros(len(self.STAGES), np.int64)
        check(lib().hpx_plan_stage_times(self._h, ctypes.c_void_p(ms.ctypes.data),
                                         ctypes.c_void_p(n.ctypes.data)), "hpx_plan_stage_times")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.STAGES)}

    def chain_stats(self) -> tuple[int, int]:
        """(active, total) (l, m, ring pair) triples of the Legendre stage."""
        a = ctypes.c_int64()
        t = ctypes.c_int64()
        check(lib().hpx_plan_chain_stats(self._h, ctypes.byref(a), ctypes.byref(t)), "hpx_plan_chain_stats")
        return int(a.value), int(t.value)

    def ring_table(self) -> dict:
        R = 4 * self.nside - 1
        start = np.zeros(R, np.int64)
        nphi = np.zeros(R, np.int32)
        z = np.zeros(R, np.float64)
        sinth = np.zeros(R, np.float64)
        sigma = np.zeros(R, np.int32)
        P = ctypes.c_void_p
        check(lib().hpx_plan_ring_table(self._h, P(start.ctypes.data), P(nphi.ctypes.data), P(z.ctypes.data),
                                        P(sinth.ctypes.data), P(sigma.ctypes.data)), "hpx_plan_ring_table")
        return {"start": start, "nphi": nphi, "z": z, "sinth": sinth, "sigma": sigma}


LAYOUTS = {"ring": _lib.HPX_RING, "nested": _lib.HPX_NESTED, "flat": _lib.HPX_FLAT}


def reorder(maps: torch.Tensor, nside: int, src: str, dst: str, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """Maps [..., 12 nside^2] on the GPU from layout src to dst (Sec. III-B,
    through the (x, y, f) representation)."""
    if not (isinstance(maps, torch.Tensor) and maps.is_cuda and maps.is_contiguous()):
        raise ValueError("maps must be a contiguous CUDA tensor")
    npix = 12 * nside * nside
    if maps.shape[-1] != npix:
        raise ValueError(f"last dimension must be {npix}")
    out = torch.empty_like(maps) if out is None else out
    nb = maps.numel() // npix
    check(lib().hpx_reorder(nside, nb, maps.element_size(), LAYOUTS[src], LAYOUTS[dst],
                            ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(_stream_handle(stream, maps.device))), "hpx_reorder")
    return out


def layout_index(nside: int, src: str, dst: str, device=None) -> torch.Tensor:
    """int64 [12 nside^2]: index[t] = the src index of the pixel whose dst index is t."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    idx = torch.empty(12 * nside * nside, dtype=torch.int64, device=device)
    check(lib().hpx_layout_index(nside, LAYOUTS[src], LAYOUTS[dst], ctypes.c_void_p(idx.data_ptr()),
                                 ctypes.c_void_p(_stream_handle(None, device))), "hpx_layout_index")
    check(lib().hpx_layout_status(), "hpx_layout_status")
    return idx


_plan_cache: dict = {}
_plan_lock = threading.Lock()


def get_plan(nside: int, lmax: int, mmax: int | None, nbatch: int, dtype: str, device=None,
             lambda_table: bool = False, tensor_cores: bool = False) -> Plan:
    """A cached plan per (geometry, batch, dtype, device, options)."""
    mmax = lmax if mmax is None else mmax
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    key = (nside, lmax, mmax, nbatch, dtype, device, lambda_table, tensor_cores)
    with _plan_lock:
        p = _plan_cache.get(key)
        if p is None:
            p = Plan(nside, lmax, mmax, nbatch, dtype, lambda_table, device, tensor_cores)
            _plan_cache[key] = p
    return p


def clear_plans() -> None:
    """Close and forget every cached plan (get_plan, the autograd functions)."""
    with _plan_lock:
        for p in _plan_cache.values():
            p.close()
        _plan_cache.clear()
