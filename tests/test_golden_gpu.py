"""The hand-derived Nside-1 and Nside-2 worked examples of tests/golden/
through every plan kind of the CUDA library: analysis (Eq. 1), synthesis
(Eq. 2) and both adjoints (Sec. III-F), against the closed forms themselves
rather than the oracle.  Bars as in the parity tests: relative L2 per
channel, FP64 1e-12, FP32 (CUDA cores, either tensor-core split scheme,
tables streamed from the host, or lambda recomputed into streamed blocks)
1e-5, and the mixed-precision bounds for the 16-bit contractions."""
import numpy as np
import pytest
import torch

import golden_cases as g

pytestmark = pytest.mark.gpu

KINDS = {
    "f64": (dict(dtype="f64"), 1e-12),
    "f64-table": (dict(dtype="f64", lambda_table=True), 1e-12),
    "f32": (dict(dtype="f32"), 1e-5),
    "f32-table": (dict(dtype="f32", lambda_table=True), 1e-5),
    "f32-tc-fp16-split": (dict(dtype="f32", lambda_table=True, tensor_cores=True), 1e-5),
    "f32-tc-tf32x3": (dict(dtype="f32", lambda_table=True, tensor_cores=True, tf32x3=True), 1e-5),
    "f32-out-of-core": (dict(dtype="f32", out_of_core=True, stage_bytes=1 << 20), 1e-5),
    "f32-streamed": (dict(dtype="f32", streamed=True, stage_bytes=1 << 20), 1e-5),
    # 16-bit contractions, at the mixed-precision bounds
    "bf16": (dict(dtype="bf16"), 1e-2),
    "fp16": (dict(dtype="fp16"), 2e-3),
    "bf16x3": (dict(dtype="bf16x3"), 1e-4),
    "fp16x3": (dict(dtype="fp16x3"), 1e-5),
}


def rel_err(got, ref):
    num = np.linalg.norm((got - ref).reshape(ref.shape[0], -1), axis=1)
    den = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    return float(np.max(num / den))


def _run(h, nside, kw, ana, syn):
    f64 = kw["dtype"] == "f64"  # every other dtype has FP32 inputs and outputs
    rt, ct = (torch.float64, torch.complex128) if f64 else (torch.float32, torch.complex64)
    maps = np.stack([c[1] for c in ana])
    alm = np.stack([c[2] for c in syn])
    out = {}
    with h.Plan(nside, g.LMAX, g.MMAX, len(ana), **kw) as p:
        dm = torch.from_numpy(maps).to(rt).cuda()
        out["map2alm"] = p.map2alm(dm)
        out["alm2map_adjoint"] = p.alm2map_adjoint(dm)
    with h.Plan(nside, g.LMAX, g.MMAX, len(syn), **kw) as p:
        da = torch.from_numpy(alm).to(ct).cuda()
        out["alm2map"] = p.alm2map(da)
        out["map2alm_adjoint"] = p.map2alm_adjoint(da)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("nside", g.NSIDES)
@pytest.mark.parametrize("kind", list(KINDS))
def test_worked_examples_on_gpu(kind, nside):
    import paper_2510_01785_gb300 as h
    kw, tol = KINDS[kind]
    ana, syn = g.analysis_cases(nside), g.synthesis_cases(nside)
    aref = np.stack([c[2] for c in ana])
    fref = np.stack([c[1] for c in syn])
    w = 4 * np.pi / (12 * nside * nside)
    got = _run(h, nside, kw, ana, syn)
    ref = {"map2alm": aref, "alm2map": fref,
           "alm2map_adjoint": aref / w,     # Y^dagger: unit weights
           "map2alm_adjoint": fref * w}     # W Y: equal weights 4 pi / Npix
    for op, r in ref.items():
        x = got[op].cpu().numpy().astype(np.complex128 if np.iscomplexobj(r) else np.float64)
        assert x.shape == r.shape, op
        e = rel_err(x, r)
        assert e <= tol, (kind, nside, op, e)
