"""hpx_plan_estimate_bytes (admission control, no allocation) against the
device bytes plans actually hold: an upper bound, and not a loose one."""
import pytest

pytestmark = pytest.mark.gpu

CASES = [  # nside, lmax, nbatch, dtype, Plan keywords, flags
    (64, 191, 4, "f64", {}, 0),
    (128, 383, 8, "f32", {}, 0),
    (128, 383, 8, "f32", dict(lambda_table=True), 1),
    (128, 383, 8, "f32", dict(lambda_table=True, tensor_cores=True), 3),
    (128, 383, 8, "f32", dict(lambda_table=True, tensor_cores=True, tf32x3=True), 11),
    (128, 383, 40, "bf16", {}, 0),
    (256, 767, 3, "fp16x3", {}, 0),
    (256, 767, 8, "f32", dict(streamed=True), 19),
    (128, 383, 8, "bf16", dict(streamed=True), 16),  # (the estimate assumes the default staging size)
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[3]}-flags{c[5]}-ns{c[0]}-b{c[2]}" for c in CASES])
def test_estimate_bounds_the_plan(case):
    import paper_2510_01785_gb300 as hpx
    from paper_2510_01785_gb300._lib import lib
    nside, lmax, nb, dtype, kw, flags = case
    est = lib().hpx_plan_estimate_bytes(nside, lmax, lmax, nb, hpx.DTYPES[dtype], flags)
    with hpx.Plan(nside, lmax, lmax, nb, dtype, **kw) as p:
        held = p.device_bytes
    print(dtype, flags, est, held, est / held)
    assert held <= est <= 2 * held
