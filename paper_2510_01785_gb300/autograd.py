"""Differentiable transforms: torch.autograd.Function wrappers over libhpx.

Sec. III-F / IV-C of arXiv 2510.01785: the gradient of the synthesis is the
adjoint synthesis and the gradient of the analysis the adjoint analysis; no
generic autodiff, and lambda_lm is recomputed by the backward call (the
forward saves only the plan, no Legendre values).

Coefficients are complex tensors of a real field (m >= 0 stored).  PyTorch
treats them as the real pairs (Re a_lm, Im a_lm), so their gradient is
dL/dRe + i dL/dIm; the library's gradient entry points apply the factors
that convention needs (2 for m >= 1, and Im a_l0 does not enter the
synthesis).
"""
from __future__ import annotations

import torch

from . import get_plan


class Alm2Map(torch.autograd.Function):
    """p = Y a; backward: dL/da = D Y^dagger dL/dp."""

    @staticmethod
    def forward(ctx, alm, plan):
        ctx.plan = plan
        return plan.alm2map(alm.contiguous())

    @staticmethod
    def backward(ctx, grad_map):
        return ctx.plan.alm2map_grad(grad_map.contiguous()), None


class Map2Alm(torch.autograd.Function):
    """a = Y^dagger W p; backward: dL/dp = W Y D^-1 dL/da."""

    @staticmethod
    def forward(ctx, maps, plan):
        ctx.plan = plan
        return plan.map2alm(maps.contiguous())

    @staticmethod
    def backward(ctx, grad_alm):
        return ctx.plan.map2alm_grad(grad_alm.contiguous()), None


def _nside(npix: int) -> int:
    nside = int(round((npix / 12) ** 0.5))
    if 12 * nside * nside != npix:
        raise ValueError(f"{npix} is not 12 nside^2")
    return nside


def map2alm(maps: torch.Tensor, lmax: int, mmax: int | None = None, lambda_table: bool = False) -> torch.Tensor:
    """Differentiable analysis of [nbatch, npix] (or [npix]) maps."""
    squeeze = maps.dim() == 1
    x = maps.unsqueeze(0) if squeeze else maps
    dtype = "f64" if x.dtype == torch.float64 else "f32"
    plan = get_plan(_nside(x.shape[1]), lmax, mmax, x.shape[0], dtype, x.device, lambda_table)
    out = Map2Alm.apply(x, plan)
    return out[0] if squeeze else out


def alm2map(alm: torch.Tensor, nside: int, lmax: int, mmax: int | None = None,
            lambda_table: bool = False) -> torch.Tensor:
    """Differentiable synthesis of [nbatch, nalm] (or [nalm]) coefficients."""
    squeeze = alm.dim() == 1
    x = alm.unsqueeze(0) if squeeze else alm
    dtype = "f64" if x.dtype == torch.complex128 else "f32"
    plan = get_plan(nside, lmax, mmax, x.shape[0], dtype, x.device, lambda_table)
    out = Alm2Map.apply(x, plan)
    return out[0] if squeeze else out
