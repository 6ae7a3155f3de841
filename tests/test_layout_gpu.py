"""RING / NESTED / FLAT reordering (Sec. III-B) on the GPU against the
oracle's geometric matching: the index maps bit for bit, and reorders of
data of every element size."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

PAIRS = [(a, b) for a in ("ring", "nested", "flat") for b in ("ring", "nested", "flat") if a != b]


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 32, 64])
def test_layout_index_matches_oracle(nside):
    import paper_2510_01785_gb300 as hpx
    for src, dst in PAIRS:
        got = hpx.layout_index(nside, src, dst).cpu().numpy()
        assert np.array_equal(got, oracle.layout_index(nside, src, dst)), (src, dst)


@pytest.mark.parametrize("nside,nb", [(1, 2), (2, 5), (16, 3), (64, 9)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.complex128])
def test_reorder_moves_data(dtype, nside, nb):
    """Every pair of layouts, against the oracle's index map: faces in one
    tile (nside <= 32) and in several tiles (64), channel counts that leave
    a remainder after the kernel's groups of four."""
    import paper_2510_01785_gb300 as hpx
    npix = 12 * nside * nside
    x = torch.randn(nb, npix, dtype=dtype, device="cuda")
    for src, dst in PAIRS:
        y = hpx.reorder(x, nside, src, dst)
        idx = torch.from_numpy(oracle.layout_index(nside, src, dst)).cuda()
        assert torch.equal(y, x[:, idx]), (src, dst)
        assert torch.equal(hpx.reorder(y, nside, dst, src), x)


def test_reorder_round_trip_nside1024():
    """At full size: ring -> nested -> flat -> ring is the identity, and
    sampled entries follow the index map."""
    import paper_2510_01785_gb300 as hpx
    nside = 1024
    x = torch.randn(2, 12 * nside * nside, device="cuda")
    n = hpx.reorder(x, nside, "ring", "nested")
    f = hpx.reorder(n, nside, "nested", "flat")
    assert torch.equal(hpx.reorder(f, nside, "flat", "ring"), x)
    idx = hpx.layout_index(nside, "ring", "nested")
    t = torch.randint(0, 12 * nside * nside, (4096,), device="cuda")
    assert torch.equal(n[:, t], x[:, idx[t]])
    assert hpx.layout_index(nside, "ring", "nested").unique().numel() == 12 * nside * nside


def test_reorder_every_pair_nside1024_sampled():
    """At full size, every pair of layouts follows the index map on sampled
    target pixels, and the reverse reorder restores the input."""
    import paper_2510_01785_gb300 as hpx
    nside = 1024
    x = torch.randn(3, 12 * nside * nside, device="cuda")
    t = torch.randint(0, 12 * nside * nside, (1 << 16,), device="cuda")
    for src, dst in PAIRS:
        y = hpx.reorder(x, nside, src, dst)
        idx = hpx.layout_index(nside, src, dst)
        assert torch.equal(y[:, t], x[:, idx[t]]), (src, dst)
        assert torch.equal(hpx.reorder(y, nside, dst, src), x), (src, dst)
