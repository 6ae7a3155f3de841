"""The oracle against hand-derived worked examples at Nside 1 and 2
(tests/golden/): the pixel centres of the grid (Sec. III-A), the analysis of
Eq. 1 and the synthesis of Eq. 2, each value a closed form written out from
the pixel centres -- including the m = 4 alias on 4-pixel rings with the sign
of their half-pixel shift, and at Nside 2 the cap rings next to the poles."""
import numpy as np
import pytest

import golden_cases as g
import oracle


@pytest.mark.parametrize("nside", g.NSIDES)
def test_pixel_centres_match_the_worked_grid(nside):
    px = g.pixels(nside)
    th, ph = oracle.pixel_angles(nside)
    assert np.max(np.abs(np.cos(th) - px[:, 0])) < 1e-15
    assert np.max(np.abs(np.sin(th) - px[:, 1])) < 1e-15
    assert np.max(np.abs(ph - px[:, 2])) < 1e-15


@pytest.mark.parametrize("tier", ["direct", "sep"])
@pytest.mark.parametrize("nside", g.NSIDES)
def test_analysis_worked_examples(nside, tier):
    cases = g.analysis_cases(nside)
    maps = np.stack([c[1] for c in cases])
    got = oracle.map2alm(maps, g.LMAX, g.MMAX, tier=tier)
    for (name, _, ref), a in zip(cases, got):
        assert np.max(np.abs(a - ref)) < 1e-14, name


@pytest.mark.parametrize("tier", ["direct", "sep"])
@pytest.mark.parametrize("nside", g.NSIDES)
def test_synthesis_worked_examples(nside, tier):
    cases = g.synthesis_cases(nside)
    alm = np.stack([c[2] for c in cases])
    got = oracle.alm2map(alm, nside, g.LMAX, g.MMAX, tier=tier)
    for (name, ref, _), f in zip(cases, got):
        assert np.max(np.abs(f - ref)) < 1e-14, name


def test_worked_examples_are_not_trivial():
    """Each case has a nonzero answer, and the aliased m = 4 appears in both
    directions at both Nside, so a dropped alias or shift cannot pass by
    zeros."""
    i44 = g.alm_index(4, 4)
    for nside in g.NSIDES:
        for _, f, a in g.analysis_cases(nside) + g.synthesis_cases(nside):
            assert np.max(np.abs(f)) > 0.1 and np.max(np.abs(a)) > 0.1
        assert any(abs(a[i44]) > 0.01 for _, _, a in g.analysis_cases(nside))
        assert any(abs(a[i44]) > 0.1 for _, _, a in g.synthesis_cases(nside))


@pytest.mark.parametrize("nside", g.NSIDES)
def test_adjoints_from_the_worked_examples(nside):
    """Sec. III-F: the adjoint of synthesis is Y^dagger, the analysis sum
    with unit weights (the worked analysis times Npix / 4 pi); the adjoint of
    analysis is W Y (the worked synthesis times 4 pi / Npix)."""
    w = 4 * np.pi / (12 * nside * nside)
    ana = g.analysis_cases(nside)
    got = oracle.alm2map_adjoint(np.stack([c[1] for c in ana]), g.LMAX, g.MMAX)
    for (name, _, ref), a in zip(ana, got):
        assert np.max(np.abs(a - ref / w)) < 1e-13, name
    syn = g.synthesis_cases(nside)
    got = oracle.map2alm_adjoint(np.stack([c[2] for c in syn]), nside, g.LMAX, g.MMAX)
    for (name, ref, _), f in zip(syn, got):
        assert np.max(np.abs(f - ref * w)) < 1e-14, name
