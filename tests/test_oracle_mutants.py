"""Planted mistakes in the oracle fail its pins.

Each case copies oracle.c, plants one plausible mistake in the copy (a
dropped sign, term, factor or offset), builds it into a temporary library
beside the test and checks that the pins catch it:
  * MUTANTS: the loader is pointed at the copy in this process and the
    hand-derived Nside-1 and Nside-2 worked examples of tests/golden/ (pixel
    centres, Eq. 1 analysis and Eq. 2 synthesis in both oracle tiers) must
    fail;
  * WIDE: the whole pin suite (test_oracle.py and the worked examples) runs
    in a subprocess against the copy (HPX_ORACLE_LIB) and must fail -- for
    mistakes that show only at larger Nside, in the log-domain chain or in
    the weighted operators.
The unmodified copy, built the same way, passes both.  The source snippet of
each mistake must occur exactly once, so that a change to oracle.c shows up
here instead of leaving a case that plants nothing.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import golden_cases as g
import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTANTS = {
    "cap ring z with 2 Nside^2 instead of 3 Nside^2 (Sec. III-A)": (
        "const double den = 3.0 * (double)(ns * ns);", "const double den = 2.0 * (double)(ns * ns);"),
    "cap ring half-pixel shift dropped (Sec. III-A)": (
        "    *sigma = 1;\n", "    *sigma = 0;\n"),
    "condon-shortley sign dropped (Eq. 15)": (
        "v = snorm(-v.mant * sqrt(", "v = snorm(v.mant * sqrt("),
    "1/alpha_{l-1} dropped from the recurrence (Eq. 16)": (
        "(l - 1 > m) ? 1.0 / alpha_lm(l - 1, m) : 0.0", "(l - 1 > m) ? 1.0 : 0.0"),
    "lambda_mm product (2k-1)/(2k) instead of (2k+1)/(2k) (Eq. 8)": (
        "sqrt((2.0 * k + 1.0) / (2.0 * k))", "sqrt((2.0 * k - 1.0) / (2.0 * k))"),
    "belt half-pixel shift parity flipped (Sec. III-A)": (
        "*sigma = (int)((i - ns + 1) & 1);", "*sigma = (int)((i - ns) & 1);"),
    "belt z without its factor 2 (Sec. III-A)": (
        "*z = (double)(2 * (2 * ns - ii)) / (double)(3 * ns);", "*z = (double)(2 * ns - ii) / (double)(3 * ns);"),
    "ring phase offset phi_0 dropped in the ring DFT (Eq. 13, 26)": (
        "(m * (2 * (int64_t)x + sigma)) % (2 * (int64_t)n)", "(m * (2 * (int64_t)x)) % (2 * (int64_t)n)"),
    "conjugation dropped in the ring DFT (Eq. 26)": (
        "acc_add(&im, -p[x] * cs[2 * r + 1]);", "acc_add(&im, p[x] * cs[2 * r + 1]);"),
    "factor 2 of the m >= 1 terms dropped in the ring synthesis (Eq. 24)": (
        "acc_add(&s, 2.0 * (F[2 * m] * cs[2 * r] - F[2 * m + 1] * cs[2 * r + 1]));",
        "acc_add(&s, (F[2 * m] * cs[2 * r] - F[2 * m + 1] * cs[2 * r + 1]));"),
    "sign of Im a_lm flipped in the direct synthesis (Eq. 24)": (
        "(a[0] * c - a[1] * sn)", "(a[0] * c + a[1] * sn)"),
}


def failures():
    """Names of the worked-example checks the loaded oracle fails."""
    bad = []
    for nside in g.NSIDES:
        px = g.pixels(nside)
        th, ph = oracle.pixel_angles(nside)
        if np.max(np.abs(np.cos(th) - px[:, 0])) > 1e-15 or np.max(np.abs(ph - px[:, 2])) > 1e-15:
            bad.append(f"pixels-{nside}")
        ana = g.analysis_cases(nside)
        maps = np.stack([c[1] for c in ana])
        ref = np.stack([c[2] for c in ana])
        syn = g.synthesis_cases(nside)
        alm = np.stack([c[2] for c in syn])
        fref = np.stack([c[1] for c in syn])
        for tier in ("direct", "sep"):
            if np.max(np.abs(oracle.map2alm(maps, g.LMAX, g.MMAX, tier=tier) - ref)) > 1e-14:
                bad.append(f"analysis-{tier}-{nside}")
            if np.max(np.abs(oracle.alm2map(alm, nside, g.LMAX, g.MMAX, tier=tier) - fref)) > 1e-14:
                bad.append(f"synthesis-{tier}-{nside}")
    return bad


def _load(monkeypatch, tmp_path, text, tag):
    src = tmp_path / f"oracle_{tag}.c"
    src.write_text(text)
    so = tmp_path / f"liboracle_{tag}.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(src), "-lm"])
    monkeypatch.setattr(oracle, "_LIB", str(so))
    monkeypatch.setattr(oracle, "build", lambda force=False: str(so))
    monkeypatch.setattr(oracle, "_lib", None)


needs_gcc = pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")


@needs_gcc
def test_unmodified_copy_passes(monkeypatch, tmp_path):
    _load(monkeypatch, tmp_path, open(SRC).read(), "control")
    assert failures() == []


@needs_gcc
@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"snippet for {name!r} must occur exactly once in oracle.c"
    _load(monkeypatch, tmp_path, text.replace(old, new), "mutant")
    assert failures(), f"no worked example catches: {name}"


# Mistakes the worked examples alone may miss (some show only at Nside >= 4,
# in the log-domain chain or in the weighted operators): each must fail the
# whole pin suite, run in a subprocess against the modified build.
WIDE = {
    "cap ring z with i instead of i^2 (Sec. III-A; the same at Nside <= 2)": (
        "*z = 1.0 - (double)(ii * ii) / den;", "*z = 1.0 - (double)(ii) / den;"),
    "cap ring sin(theta) from 6 Nside^2 + i^2 (Sec. III-A)": (
        "sqrt((double)(6 * ns * ns - ii * ii))", "sqrt((double)(6 * ns * ns + ii * ii))"),
    "alpha_lm with l^2 + m^2 (Eq. 16)": (
        "return sqrt((4.0 * ld * ld - 1.0) / (ld * ld - md * md));",
        "return sqrt((4.0 * ld * ld - 1.0) / (ld * ld + md * md));"),
    "belt ring start one ring late (Sec. III-A)": (
        "*start = 2 * ns * (ns - 1) + 4 * ns * (i - ns);", "*start = 2 * ns * (ns - 1) + 4 * ns * (i - ns + 1);"),
    "south cap start with (i - 1) for (i + 1) (Sec. III-A)": (
        "npix - 2 * ii * (ii + 1)", "npix - 2 * ii * (ii - 1)"),
    "direct analysis without the ring weights (Eq. 1, 26)": (
        "const double lw = lam[((size_t)m * g.nring + y) * L + l] * (w ? w[y] : 1.0);",
        "const double lw = lam[((size_t)m * g.nring + y) * L + l];"),
    "separable synthesis without the per-ring scale (W Y, Sec. III-F)": (
        "out[(size_t)b * nout + ooff[k] + x] = acc_val(&s) * (scale ? scale[y] : 1.0);",
        "out[(size_t)b * nout + ooff[k] + x] = acc_val(&s);"),
    "log2 lambda without its binary exponent (Eq. 8 below the double range)": (
        ": log2(fabs(p1.mant)) + (double)p1.ex;", ": log2(fabs(p1.mant));"),
    "sign of the lambda_{l-2} term of the recurrence (Eq. 16)": (
        "ainv_prev * ldexp(p2.mant, p2.ex - e);", "(-ainv_prev) * ldexp(p2.mant, p2.ex - e);"),
}
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle.py", "tests/test_oracle_golden.py"]


def _build(tmp_path, text, tag):
    src = tmp_path / f"oracle_{tag}.c"
    src.write_text(text)
    so = tmp_path / f"liboracle_{tag}.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(src), "-lm"])
    return so


def _pins_pass(so):
    env = dict(os.environ, HPX_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode == 0, r.stdout[-1500:]


@needs_gcc
def test_unmodified_copy_passes_the_pin_suite(tmp_path):
    ok, out = _pins_pass(_build(tmp_path, open(SRC).read(), "control"))
    assert ok, out


@needs_gcc
@pytest.mark.parametrize("name", list(WIDE))
def test_planted_mistake_fails_the_pin_suite(name, tmp_path):
    old, new = WIDE[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"snippet for {name!r} must occur exactly once in oracle.c"
    ok, _ = _pins_pass(_build(tmp_path, text.replace(old, new), "mutant"))
    assert not ok, f"no pin catches: {name}"
