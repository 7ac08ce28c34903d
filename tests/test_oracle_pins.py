"""Pins of the FP64 CPU oracle against things other than itself: values the
paper prints, closed forms, library routines, invariants and brute force."""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W
from tests.golden import printed_values

LN2 = math.log(2.0)


# --------------------------------------------------------------------------
# Philox4x32-10 against PyTorch's open-source engine (run as a library)
# --------------------------------------------------------------------------
_PHILOX_HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::Philox4_32 e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def test_philox_matches_pytorch_engine():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) or not shutil.which("g++"):
        pytest.skip("torch headers or g++ unavailable")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "h.cpp"), os.path.join(d, "h")
    open(src, "w").write(_PHILOX_HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I" + inc, src, "-o", exe], check=True)
    rng = np.random.default_rng(7)
    cases = [(0, 0, 0), (2**64 - 1, 2**64 - 1, 2**64 - 1)]
    for _ in range(300):
        cases.append(tuple(int(x) for x in rng.integers(0, 2**63, size=3, dtype=np.int64) * 2 + 1))
    inp = "".join("%d %d %d\n" % c for c in cases)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (seed, sub, off), line in zip(cases, out):
        # engine: key = seed, counter = (off_lo, off_hi, sub_lo, sub_hi)
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert ob.philox(ctr, key) == [int(x) for x in line.split()]


def test_philox_uniformity_and_independence():
    # chi-square of the top byte over 2^16 blocks and no equal neighbours
    words = np.array([ob.philox([i, 0, 5, 0], [1, 0]) for i in range(20000)], dtype=np.uint64)
    hist = np.bincount((words.ravel() >> 24).astype(np.int64), minlength=256)
    chi2 = ((hist - hist.mean()) ** 2 / hist.mean()).sum()
    assert stats.chi2.sf(chi2, 255) > 1e-4


# --------------------------------------------------------------------------
# intrinsic rocking curve
# --------------------------------------------------------------------------
def test_pv_total_width_matches_printed_values():
    pv = printed_values()
    F, _ = ob.pv_width(50.0, 8.0)
    assert abs(F - pv["pv_total_fwhm_50_8"][0]) < 0.05
    F, _ = ob.pv_width(100.0, 20.0)
    assert abs(F - pv["pv_total_fwhm_100_20"][0]) < 0.05


def test_pv_limits():
    F, eta = ob.pv_width(7.0, 0.0)
    assert F == pytest.approx(7.0, rel=1e-14) and eta == 0.0
    F, eta = ob.pv_width(0.0, 3.0)
    assert F == pytest.approx(3.0, rel=1e-14) and eta == pytest.approx(1.0, abs=1e-5)


def _spec(**kw):
    s = W.flat_hopg_mono()["spec"]
    s = dict(s)
    s.update(kw)
    return s


@pytest.mark.parametrize("irc,extra", [
    ("darwin", {}), ("darwin_prins", {"prins_g": 0.05}), ("darwin_prins", {"prins_g": 0.3}),
    ("gaussian", {}), ("lorentzian", {}), ("box", {}),
    ("pseudo_voigt", {"irc_fwhm_rad": 50e-6, "irc_lorentz_fwhm_rad": 8e-6})])
def test_irc_unit_area(irc, extra):
    kw = {"irc_fwhm_rad": 20e-6}
    kw.update(extra)
    s = _spec(irc=irc, **kw)
    f = lambda x: ob.irc(s, x)[0]
    w = s["irc_fwhm_rad"]
    pts = [-0.6 * w, -0.5 * w, 0.0, 0.5 * w, 0.6 * w]
    core = integrate.quad(f, -50 * w, 50 * w, points=pts, limit=400, epsabs=0, epsrel=1e-11)[0]
    tails = 2 * integrate.quad(f, 50 * w, np.inf, limit=400, epsabs=0, epsrel=1e-9)[0]
    assert core + tails == pytest.approx(1.0, rel=2e-7)


def test_darwin_integral_and_fwhm():
    # textbook: integral of the Darwin curve over y is 8/3; FWHM = (3/sqrt2) delta
    assert ob.darwin_prins_area(0.0) == pytest.approx(8.0 / 3.0, rel=1e-10)
    s = _spec(irc="darwin", irc_fwhm_rad=20e-6)
    half = ob.irc(s, 10e-6)[0]
    assert half == pytest.approx(0.5 * ob.irc_max(s), rel=1e-12)
    # plateau edge y = 1 at delta = FWHM sqrt2/3
    d = 20e-6 * math.sqrt(2) / 3
    assert ob.irc(s, 0.999999 * d)[0] == pytest.approx(ob.irc_max(s), rel=1e-15)


def test_darwin_prins_properties():
    for g in (1e-7, 0.05, 0.3):
        s = _spec(irc="darwin_prins", irc_fwhm_rad=20e-6, prins_g=g)
        d = 20e-6 * math.sqrt(2) / 3
        A = ob.darwin_prins_area(g)
        y = np.linspace(-4, 4, 2001)
        R = ob.irc(s, y * d) * d * A
        assert np.all(R <= 1 + 1e-12)
        assert np.allclose(R, R[::-1], rtol=1e-12)
        assert R.max() == pytest.approx(R[1000], rel=1e-12)        # peak at the centre
        assert R[1000] == pytest.approx((math.sqrt(1 + g * g) - g) ** 2, rel=1e-12)
    # g -> 0 reduces to the Darwin curve
    s0 = _spec(irc="darwin", irc_fwhm_rad=20e-6)
    s1 = _spec(irc="darwin_prins", irc_fwhm_rad=20e-6, prins_g=1e-9)
    x = np.linspace(-60e-6, 60e-6, 301)
    assert np.allclose(ob.irc(s0, x), ob.irc(s1, x), rtol=1e-6)


def test_gaussian_lorentzian_irc_equal_library_pdfs():
    s = _spec(irc="gaussian", irc_fwhm_rad=30e-6)
    x = np.linspace(-80e-6, 80e-6, 41)
    sig = 30e-6 / (2 * math.sqrt(2 * LN2))
    assert np.allclose(ob.irc(s, x), stats.norm.pdf(x, scale=sig), rtol=1e-12)
    s = _spec(irc="lorentzian", irc_fwhm_rad=30e-6)
    assert np.allclose(ob.irc(s, x), stats.cauchy.pdf(x, scale=15e-6), rtol=1e-12)


# --------------------------------------------------------------------------
# mosaic distribution on the sphere
# --------------------------------------------------------------------------
def _closed_form_quantile(mdf, G, u, comp=None):
    """Closed-form inverse CDFs of q = 1 - cos(theta) (derived in the design notes)."""
    if comp is None:
        comp = 1.0 - u
    if mdf == "vmf":
        s2 = (G / (2 * math.sqrt(2 * LN2))) ** 2
        # 1 - F = (exp(-q/s^2) - exp(-2/s^2)) / (1 - exp(-2/s^2))
        return -s2 * math.log(comp * (1 - math.exp(-2 / s2)) + math.exp(-2 / s2))
    if mdf == "wl":
        a2 = G * G / 4
        return 0.5 * a2 * math.expm1((1 - comp) * math.log1p(4 / a2))
    if mdf == "swl":
        b = 2 * math.sinh(G / 4) ** 2
        return 1.0 / (1.0 / b - (1 - comp) * (1.0 / b - 1.0 / (b + 2))) - b
    if mdf == "uniform":
        return (1 - comp) * 2 * math.sin(G / 4) ** 2
    raise ValueError(mdf)


@pytest.mark.parametrize("mdf", ["vmf", "wl", "swl", "uniform"])
@pytest.mark.parametrize("G_deg", [0.06, 0.4, 1.3])
def test_mdf_table_equals_closed_form_quantiles(mdf, G_deg):
    G = G_deg * W.DEG
    s = _spec(mdf=mdf, mdf_fwhm_rad=G)
    t = ob.mdf_table(s)
    body = np.array(t.body)
    for i in list(range(0, 4096, 97)) + [1, 4094, 4095]:
        want = _closed_form_quantile(mdf, G, i / 4096.0)
        assert body[i] == pytest.approx(want, rel=1e-10, abs=1e-300)
    tail = np.array(t.tail)
    for j in (0, 1, 37, 128, 200, 255, 256):
        comp = 2.0 ** -(12 + 21 * j / 256)
        want = _closed_form_quantile(mdf, G, None, comp=comp)
        assert tail[j] == pytest.approx(want, rel=1e-9)


def test_mdf_sphere_normalisations_printed_in_paper():
    G = 0.1 * W.DEG
    # Eq. (MF): normalisation 2 pi s^2 (1 - exp(-2/s^2)) for exp((cos th - 1)/s^2)
    s2 = (G / (2 * math.sqrt(2 * LN2))) ** 2
    assert 2 * math.pi * ob.mdf_norm(_spec(mdf="vmf", mdf_fwhm_rad=G)) == pytest.approx(
        2 * math.pi * s2 * (1 - math.exp(-2 / s2)), rel=1e-12)
    # Eq. (WL): normalisation pi ln(1 + (4/Gamma)^2)
    assert 2 * math.pi * ob.mdf_norm(_spec(mdf="wl", mdf_fwhm_rad=G)) == pytest.approx(
        math.pi * math.log1p((4 / G) ** 2), rel=1e-12)
    # Eq. (SWL): 4 pi / sinh^2(Gamma/2) for 1/(cosh(Gamma/2) - cos th)^2
    assert 2 * math.pi * ob.mdf_norm(_spec(mdf="swl", mdf_fwhm_rad=G)) == pytest.approx(
        4 * math.pi / math.sinh(G / 2) ** 2, rel=1e-10)


def test_gaussian_mdf_small_width_is_rayleigh():
    # for Gamma << 1 the polar angle of a Gaussian sphere density is Rayleigh:
    # F(theta) = 1 - exp(-4 ln2 theta^2 / Gamma^2)
    G = 1e-4
    s = _spec(mdf="gaussian", mdf_fwhm_rad=G)
    t = ob.mdf_table(s)
    body = np.array(t.body)
    for i in (1, 100, 1000, 2048, 3000, 4000, 4095):
        u = i / 4096.0
        th = G * math.sqrt(-math.log(1 - u) / (4 * LN2))
        q = 2 * math.sin(th / 2) ** 2
        assert body[i] == pytest.approx(q, rel=1e-7)


def test_lorentzian_mdf_shape_ratio():
    # small-angle CDF of sin(th)/(a^2+th^2): proportional to ln(1 + th^2/a^2)
    G = 0.05 * W.DEG
    a = G / 2
    s = _spec(mdf="lorentzian", mdf_fwhm_rad=G)
    th1, th2 = 0.5 * G, 3 * G
    F1 = ob.mdf_cdf(s, 2 * math.sin(th1 / 2) ** 2)
    F2 = ob.mdf_cdf(s, 2 * math.sin(th2 / 2) ** 2)
    assert F1 / F2 == pytest.approx(math.log1p((th1 / a) ** 2) / math.log1p((th2 / a) ** 2), rel=1e-5)


def test_mdf_table_lookup_interpolates_knots():
    s = _spec(mdf="gaussian", mdf_fwhm_rad=0.4 * W.DEG)
    t = ob.mdf_table(s)
    body = np.array(t.body)
    for i in (0, 5, 2000, 4093):
        w_lo = (i << 20)
        got = ob.mdf_table_lookup(t, [w_lo, w_lo | 0xFFFFF])
        f0, f1 = 0.5 / 2**20, (0xFFFFF + 0.5) / 2**20
        assert got[0] == pytest.approx(body[i] + f0 * (body[i + 1] - body[i]), rel=1e-15)
        assert got[1] == pytest.approx(body[i] + f1 * (body[i + 1] - body[i]), rel=1e-15)
    # tail: the largest word maps to 1 - u = 2^-33, tau = 33
    assert ob.mdf_table_lookup(t, [0xFFFFFFFF])[0] == pytest.approx(t.tail[256], rel=1e-15)
    # monotone everywhere
    ws = np.sort(np.random.default_rng(1).integers(0, 2**32, 20000, dtype=np.uint64))
    q = ob.mdf_table_lookup(t, ws)
    assert np.all(np.diff(q) >= 0)


def test_mdf_table_error_bound_against_exact_inverse():
    s = _spec(mdf="pseudo_voigt", mdf_fwhm_rad=0.1 * W.DEG, mdf_eta=0.5)
    t = ob.mdf_table(s)
    rng = np.random.default_rng(3)
    for w in rng.integers(0, 0xFFF00000, 12, dtype=np.uint64):
        u = (int(w) + 0.5) / 2**32
        exact = ob.mdf_quantile_exact(s, u)
        table = ob.mdf_table_lookup(t, [int(w)])[0]
        assert table == pytest.approx(exact, rel=2e-3)


# --------------------------------------------------------------------------
# per-ray constants
# --------------------------------------------------------------------------
def test_bragg_law_constants():
    s = _spec()
    for E in (5.0, 8.0, 12.0):
        c = ob.ray_constants(s, E)
        lam = 12.398419843320026 / E
        assert 2 * 3.354 * math.sin(c["alpha_B"]) == pytest.approx(lam, rel=1e-15)
        assert c["mubar"] == pytest.approx(c["mu0"] + c["Q"] * ob.irc_max(s), rel=1e-15)
    c = ob.ray_constants(s, 1.5)        # hc/E > 2d: no Bragg reflection possible
    assert c["no_bragg"] == 1 and c["Q"] == 0.0 and c["p_abs"] == 1.0


def test_appendix_bragg_angle_is_graphite_at_8_5_keV():
    # the appendix's alpha_B = 0.2192 rad is graphite (002) near 8.5 keV
    c = ob.ray_constants(_spec(), 8.5)
    assert c["alpha_B"] == pytest.approx(printed_values()["appendix_alpha_B"][0], abs=1e-4)


# --------------------------------------------------------------------------
# the reflectivity constant Q (Sec. 2.2.3, Eq. ZachReflXsec) from a Darwin width
# --------------------------------------------------------------------------
R_E_MM = 2.8179403262e-12          # classical electron radius (CODATA 2018), mm


def test_reflectivity_constant_of_the_flat_hopg_workload():
    """The flat HOPG workload gives its reflection strength as a Darwin FWHM of 20 urad
    at 8 keV on graphite (002).  Two textbook relations of the kinematic/dynamical
    theory fix Q from it, independently of how the oracle arranges them: the Darwin
    curve's total-reflection plateau has half-width delta = r_e lambda^2 |F| / (pi V
    sin 2 aB) (Darwin; Zachariasen; Als-Nielsen & McMorrow, ch. 6) and FWHM
    3 delta / sqrt(2) (the curve (|y| - sqrt(y^2 - 1))^2 halves at |y| = 3 / (2 sqrt 2));
    the mosaic cross-section constant is Q = |r_e F / V|^2 lambda^3 / sin 2 aB (Sec.
    2.2.3, Eq. ZachReflXsec).  Hence delta = 9.43 urad and Q = 2.54e-3 / mm, the
    value written down from these relations before the oracle existed."""
    w = W.flat_hopg_mono()
    c = ob.ray_constants(w["spec"], 8.0)
    lam_mm = 12.398419843320026 / 8.0 * 1e-7
    s2 = math.sin(2.0 * math.asin(lam_mm * 1e7 / (2.0 * 3.354)))
    delta = 20e-6 / (3.0 / math.sqrt(2.0))
    F_over_V = delta * math.pi * s2 / (R_E_MM * lam_mm ** 2)       # |F| / V, mm^-3
    Q = (R_E_MM * F_over_V) ** 2 * lam_mm ** 3 / s2
    assert delta == pytest.approx(9.43e-6, rel=1e-3)
    assert Q == pytest.approx(2.54e-3, rel=3e-3)
    assert c["Q"] == pytest.approx(Q, rel=1e-12)
    # the same constant given directly as K = |r_e F / V| reproduces it
    direct = dict(w["spec"], refl_K_per_mm2=R_E_MM * F_over_V)
    assert ob.ray_constants(direct, 8.0)["Q"] == pytest.approx(Q, rel=1e-12)


def test_reflectivity_constant_scales_as_lambda_cubed_over_sin_2_theta():
    # F_H does not depend on the energy in this model, so Q(E) = K^2 lambda^3 / sin 2 aB(E)
    s = W.flat_hopg_mono()["spec"]
    E = [6.5, 8.0, 11.0]
    Q = [ob.ray_constants(s, e)["Q"] for e in E]
    for e, q in zip(E[1:], Q[1:]):
        lam0, lam = 12.398419843320026 / E[0], 12.398419843320026 / e
        s0 = math.sin(2.0 * math.asin(lam0 / (2.0 * 3.354)))
        s1 = math.sin(2.0 * math.asin(lam / (2.0 * 3.354)))
        assert q / Q[0] == pytest.approx((lam / lam0) ** 3 * s0 / s1, rel=1e-12)
    # the majorant carries Q R_max (R of unit area peaks at its maximum)
    c = ob.ray_constants(s, 8.0)
    assert c["mubar"] == pytest.approx(c["mu0"] + c["Q"] * ob.irc_max(s), rel=1e-12)
