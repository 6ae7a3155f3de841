"""The oracle against hand-derived worked examples at Nside 1 (tests/golden/):
the pixel centres of the grid (Sec. III-A), the analysis of Eq. 1 for five
maps and the synthesis of Eq. 2 for five coefficient sets, each value a
closed form written out from the 12 pixel centres (including the m = 4
alias on 4-pixel rings and the half-pixel shift of rings 1 and 3)."""
import numpy as np
import pytest

import golden_cases as g
import oracle


def test_pixel_centres_match_the_worked_grid():
    px = g.pixels()
    th, ph = oracle.pixel_angles(g.NSIDE)
    assert np.max(np.abs(np.cos(th) - px[:, 0])) < 1e-15
    assert np.max(np.abs(np.sin(th) - px[:, 1])) < 1e-15
    assert np.max(np.abs(ph - px[:, 2])) < 1e-15


@pytest.mark.parametrize("tier", ["direct", "sep"])
def test_analysis_worked_examples(tier):
    cases = g.analysis_cases()
    maps = np.stack([c[1] for c in cases])
    got = oracle.map2alm(maps, g.LMAX, g.MMAX, tier=tier)
    for (name, _, ref), a in zip(cases, got):
        assert np.max(np.abs(a - ref)) < 1e-14, name


@pytest.mark.parametrize("tier", ["direct", "sep"])
def test_synthesis_worked_examples(tier):
    cases = g.synthesis_cases()
    alm = np.stack([c[2] for c in cases])
    got = oracle.alm2map(alm, g.NSIDE, g.LMAX, g.MMAX, tier=tier)
    for (name, ref, _), f in zip(cases, got):
        assert np.max(np.abs(f - ref)) < 1e-14, name


def test_worked_examples_are_not_trivial():
    """Each case has a nonzero answer, and the aliased m = 4 appears in both
    directions, so a dropped alias or shift cannot pass by zeros."""
    for _, f, a in g.analysis_cases() + g.synthesis_cases():
        assert np.max(np.abs(f)) > 0.1 and np.max(np.abs(a)) > 0.1
    i44 = g.alm_index(4, 4)
    assert any(abs(a[i44]) > 0.1 for _, _, a in g.analysis_cases())
    assert any(abs(a[i44]) > 0.1 for _, _, a in g.synthesis_cases())


def test_adjoints_from_the_worked_examples():
    """Sec. III-F: the adjoint of synthesis is Y^dagger, the analysis sum
    with unit weights (the worked analysis times Npix / 4 pi = 3 / pi); the
    adjoint of analysis is W Y (the worked synthesis times pi / 3)."""
    ana = g.analysis_cases()
    got = oracle.alm2map_adjoint(np.stack([c[1] for c in ana]), g.LMAX, g.MMAX)
    for (name, _, ref), a in zip(ana, got):
        assert np.max(np.abs(a - ref * 3 / np.pi)) < 1e-14, name
    syn = g.synthesis_cases()
    got = oracle.map2alm_adjoint(np.stack([c[2] for c in syn]), g.NSIDE, g.LMAX, g.MMAX)
    for (name, ref, _), f in zip(syn, got):
        assert np.max(np.abs(f - ref * np.pi / 3)) < 1e-14, name
