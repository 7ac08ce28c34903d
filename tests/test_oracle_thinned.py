"""Pins of the thinned candidate sampler against the plain one.

The thinned walk splits the scatter candidates by their marks (marking
theorem) and never generates those that provably cannot reflect, so it must
sample exactly the same distribution of ray paths as the plain majorant walk,
which is pinned to quadrature and closed forms elsewhere.  Checked here:
  * segments near the Bragg angle keep the plain candidate stream: records are
    identical to the plain walk's, word for word;
  * fans of directions 8 mrad either side of the Bragg angle (where thinning
    acts): the reflection probability per angle bin, the absorption
    probability and depth and the exit angles agree between the samplers
    (two-sample z and KS tests on independent streams), for every mosaic
    distribution and rocking curve;
  * the workloads' tallies and detector profiles agree (z, chi-square);
  * the first-reflection probability of the thinned walk equals the quadrature
    of Eq. (ReflXsection);
  * thinning removes most candidates off the Bragg angle."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

Z = 4.5


def flat(**kw):
    s = dict(W.flat_hopg_mono()["spec"])
    s.update(kw)
    return s


def pencil(alpha, E=8.0, dist=300.0):
    ca, sa = math.cos(alpha), math.sin(alpha)
    return dict(components=[dict(kind="mono", e0_keV=E, weight=1.0)],
                origin_mm=[-dist * ca, 0.0, dist * sa], axis=[ca, 0.0, -sa],
                cone_half_angle_rad=0.0, spot_fwhm_mm=(0.0, 0.0))


def _z(a, b, n):
    """two-sample z for binomial counts a, b out of n each"""
    p = (a + b) / (2 * n)
    return (a - b) / math.sqrt(max(2 * n * p * (1 - p), 1e-12))


def test_near_bragg_segments_keep_the_plain_stream():
    # the entry segment of a pencil 0.02 mrad off Bragg (inside X* = 37.7 urad: the Darwin tail
    # 1 / (4 y^2) reaches v* = 2^-6 at y = 4) is plain in both walks:
    # the same words give the same candidates up to the first reflection
    # (after it the reflected segment may be thinned)
    s = flat()
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    src = pencil(aB + 2e-5)
    _, tp, rp = ob.trace(dict(s, sampler="plain"), src, 20_000, seed=3, records=True)
    _, tt, rt = ob.trace(dict(s, sampler="thinned"), src, 20_000, seed=3, records=True)
    assert np.array_equal(rp["nrefl"] == 0, rt["nrefl"] == 0)
    same = rp["nrefl"] == 0
    assert same.sum() > 1000 and (~same).sum() > 100
    for f in ("outcome", "ncoll", "ix", "iy"):
        assert np.array_equal(rp[f][same], rt[f][same]), f
    assert np.array_equal(rp["pos"][same], rt["pos"][same])


CASES = [
    ("gaussian", "darwin", {}),
    ("lorentzian", "darwin_prins", {"mdf_fwhm_rad": 0.1 * W.DEG, "prins_g": 0.05}),
    ("pseudo_voigt", "pseudo_voigt", {"mdf_fwhm_rad": 0.2 * W.DEG, "mdf_eta": 0.5,
                                      "irc_fwhm_rad": 50e-6, "irc_lorentz_fwhm_rad": 8e-6}),
    ("vmf", "gaussian", {"mdf_fwhm_rad": 0.3 * W.DEG, "irc_fwhm_rad": 30e-6}),
    ("wl", "lorentzian", {"mdf_fwhm_rad": 0.1 * W.DEG, "irc_fwhm_rad": 15e-6}),
    ("swl", "darwin", {"mdf_fwhm_rad": 0.1 * W.DEG}),
    ("uniform", "box", {"mdf_fwhm_rad": 0.8 * W.DEG, "irc_fwhm_rad": 40e-6}),
]


@pytest.mark.parametrize("mdf,irc,extra", CASES)
def test_off_bragg_beams_agree_between_samplers(mdf, irc, extra):
    # a 1-D fan of directions from 8 mrad below to 8 mrad above the Bragg angle
    # (mostly thinned segments), mono 8 keV
    s = flat(mdf=mdf, irc=irc, thickness_mm=0.1, **extra)
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    n = 200_000
    rng = np.random.default_rng(7)
    a = aB + rng.uniform(-8e-3, 8e-3, n)
    dist = 300.0
    rays = dict(ox=-dist * np.cos(a), oy=np.zeros(n), oz=dist * np.sin(a),
                kx=np.cos(a), ky=np.zeros(n), kz=-np.sin(a), E=np.full(n, 8.0))
    _, _, tp, rp = ob.trace_rays(dict(s, sampler="plain"), rays, seed=5, records=True)
    _, _, tt, rt = ob.trace_rays(dict(s, sampler="thinned"), rays, seed=6, records=True)
    for key in ("absorbed", "exit_front", "exit_back"):
        assert abs(_z(tp[key], tt[key], n)) < Z, (key, tp[key], tt[key])
    for h in range(1, 3):
        assert abs(_z(tp["refl_hist"][h], tt["refl_hist"][h], n)) < Z, (h, tp["refl_hist"], tt["refl_hist"])
    # the reflection probability as a function of the offset from Bragg
    bins = np.linspace(-8e-3, 8e-3, 9)
    for lo, hi in zip(bins[:-1], bins[1:]):
        sel = (a - aB >= lo) & (a - aB < hi)
        x, y = np.count_nonzero(rp["nrefl"][sel] > 0), np.count_nonzero(rt["nrefl"][sel] > 0)
        assert abs((x - y) / math.sqrt(x + y + 1)) < Z, (lo, x, y)
    # absorption depth and reflected exit angles
    da = -rp["pos"][rp["outcome"] == 1][:, 2]
    db = -rt["pos"][rt["outcome"] == 1][:, 2]
    assert stats.ks_2samp(da, db).pvalue > 1e-4
    ra = rp["dir"][rp["outcome"] == 2][:, 0]
    rb = rt["dir"][rt["outcome"] == 2][:, 0]
    if min(len(ra), len(rb)) > 30:
        assert stats.ks_2samp(ra, rb).pvalue > 1e-4
    # the thinned walk draws far fewer candidates
    assert tt["collisions"] * 2 < tp["collisions"], (tt["collisions"], tp["collisions"])


@pytest.mark.parametrize("name", ["flat_hopg_mono", "von_hamos_hapg", "von_hamos_large"])
def test_workload_tallies_and_profiles_agree(name):
    w = getattr(W, name)()
    n = 300_000
    ip, tp, _ = ob.trace(dict(w["spec"], sampler="plain"), w["source"], n, seed=11)
    it, tt, _ = ob.trace(dict(w["spec"], sampler="thinned"), w["source"], n, seed=12)
    for key in ("miss", "absorbed", "exit_front", "exit_back", "exit_side", "det_hits"):
        assert abs(_z(tp[key], tt[key], n)) < Z, (key, tp[key], tt[key])
    # dispersive profiles in 64 blocks of columns
    blk = ip.shape[1] // 64
    c0 = ip.sum(axis=0).reshape(-1, blk).sum(axis=1)
    c1 = it.sum(axis=0).reshape(-1, blk).sum(axis=1)
    m = (c0 + c1) >= 10
    assert m.sum() >= 3
    K1, K2 = c0[m].sum(), c1[m].sum()
    chi = np.sum((math.sqrt(K2 / K1) * c0[m] - math.sqrt(K1 / K2) * c1[m]) ** 2 / (c0[m] + c1[m]))
    assert stats.chi2.sf(chi, m.sum() - 1) > 1e-3
    assert tt["collisions"] < tp["collisions"] / 3


def test_thinned_first_reflection_probability_matches_quadrature():
    # thin slab, pencil 1.5 mrad off Bragg: P(reflect before leaving) vs the
    # 2-D quadrature rate of Eq. (ReflXsection) over the path, with absorption
    s = flat(mdf="gaussian", thickness_mm=0.02, max_reflections=1)
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + 1.5e-3
    r = ob.reflection_rate(s, 8.0, a)               # per mm of path
    L = 0.02 / math.sin(a)
    mu = c["mu0"]
    # first event along the path: reflection at rate r, absorption at mu0
    p_refl = r / (r + mu) * (1 - math.exp(-(r + mu) * L))
    n = 2_000_000
    _, t, _ = ob.trace(dict(s, sampler="thinned"), pencil(a), n, seed=17)
    got = n - t["refl_hist"][0]
    sd = math.sqrt(n * p_refl * (1 - p_refl))
    assert abs(got - n * p_refl) < Z * sd, (got, n * p_refl)
