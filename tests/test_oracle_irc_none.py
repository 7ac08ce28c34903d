"""Pins of the walk without a rocking curve (Sec. 2.2.1: the IRC may be
"none"; Eq. ReflXsection with R(Delta) = delta(Delta)).

With R a delta function only crystallites at exactly a~0 = aB + Delta_M
reflect.  Pinned against what the paper and the geometry fix:

* Bragg's law holds exactly on every reflection: k_in . k_out = cos 2 a~0
  (flat and cylindrical crystals, with a peak shift, and per order);
* the reflection rate equals Q cos a~0 G(a~0) times the MDF integrated along
  the Bragg cone, computed here by a quadrature of the MDF's formula and, for
  the von Mises-Fisher MDF, by the closed form with the Bessel function I0;
* the thin-slab first-reflection probability of the walk matches that rate;
* the limit of ever narrower box rocking curves (sampled by the ordinary
  walk) gives the same reflection probability;
* two orthogonal polarisations reflect twice as often as unpolarised rays;
* the thinned sampler (per straight segment, the MDF at the smallest tilt
  each cone can reach bounds that cone, and on the facing cone a window in
  the azimuth outside which the MDF is below v* f(0)) agrees with the plain
  one (the bound f(0) for both cones) and draws far fewer candidates; with a
  narrow mosaic, where the window carries nearly all of the bound, its
  thin-slab probability still follows the cone quadrature."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

LN2 = math.log(2.0)


def flat(**kw):
    s = dict(W.flat_hopg_mono()["spec"], irc="none", refl_K_per_mm2=1.5e10, mdf="gaussian",
             mdf_fwhm_rad=0.35, thickness_mm=0.002, max_reflections=1)
    s.update(kw)
    return s


def pencil(alpha, E=8.0, dist=300.0, pol=None):
    ca, sa = math.cos(alpha), math.sin(alpha)
    src = dict(components=[dict(kind="mono", e0_keV=E, weight=1.0)],
               origin_mm=[-dist * ca, 0.0, dist * sa], axis=[ca, 0.0, -sa],
               cone_half_angle_rad=0.0, spot_fwhm_mm=(0.0, 0.0))
    if pol is not None:
        src["polarization"] = pol
    return src


def gauss_W(theta, fwhm):
    return np.exp(-4.0 * LN2 * theta ** 2 / fwhm ** 2)


def cone_rate(Q, a0, alpha, W, far=True):
    """Q cos a0 G(a0) sum over the cones of int_0^2pi f(theta(psi)) dpsi, with
    cos theta = +/- sin(alpha) sin(a0) + cos(alpha) cos(a0) cos(psi) (the
    crystallite normal on the cone about k at grazing angle alpha) and
    f = W / int W dOmega; W(theta) a function of the tilt angle"""
    Z = 2.0 * math.pi * integrate.quad(lambda t: W(t) * math.sin(t), 0.0, math.pi, limit=400,
                                       epsabs=0, epsrel=1e-12)[0]
    tot = 0.0
    for sg in ((1.0, -1.0) if far else (1.0,)):
        S, C = sg * math.sin(alpha) * math.sin(a0), math.cos(alpha) * math.cos(a0)

        def f(psi):
            return W(math.acos(max(-1.0, min(1.0, S + C * math.cos(psi))))) / Z

        tot += 2.0 * integrate.quad(f, 0.0, math.pi, limit=400, epsabs=0, epsrel=1e-11,
                                    points=[1e-3, 1e-2, 0.1])[0]
    G = 0.5 * (1.0 + math.cos(2 * a0) ** 2)
    return Q * math.cos(a0) * G * tot


def slab_probability(r, mu, L):
    return r / (r + mu) * (1.0 - math.exp(-(r + mu) * L))


def reflected_dirs(spec, src, n, seed):
    _, t, rec = ob.trace(spec, src, n, seed, records=True)
    one = rec["nrefl"] == 1
    return t, rec, rec["dir"][one]


@pytest.mark.parametrize("sampler", ["thinned", "plain"])
@pytest.mark.parametrize("shift", [0.0, 3e-4])
def test_bragg_law_on_every_reflection_flat(shift, sampler):
    s = flat(irc_shift_rad=shift, sampler=sampler)
    c = ob.ray_constants(s, 8.0)
    a0 = c["alpha_B"] + shift
    a = a0 + 0.05
    t, _, d = reflected_dirs(s, pencil(a), 40_000, 3)
    assert len(d) > 500
    k0 = np.array([math.cos(a), 0.0, -math.sin(a)])
    assert np.max(np.abs(d @ k0 - math.cos(2 * a0))) < 1e-12


def test_bragg_law_on_every_reflection_cylinder_and_orders():
    w = W.von_hamos_hapg()
    # the pencil meets the cylinder at 0.2335 rad; at 11.6 keV the orders reflect at 0.160 and 0.324 rad,
    # both within reach of a 0.35 rad wide mosaic
    s = dict(w["spec"], irc="none", mdf="gaussian", mdf_fwhm_rad=0.35, max_reflections=1, refl_K_per_mm2=1.5e10,
             orders=[(1, 1.0, 1.0), (2, 0.8, 1.0)])
    src = dict(w["source"], components=[dict(kind="mono", e0_keV=11.6, weight=1.0)], cone_half_angle_rad=0.0,
               spot_fwhm_mm=(0.0, 0.0))
    c = ob.ray_constants(s, 11.6)
    t, rec, d = reflected_dirs(s, src, 40_000, 4)
    k0 = np.asarray(src["axis"], float)
    k0 /= np.linalg.norm(k0)
    cosang = d @ k0
    targets = np.cos(2 * np.array(c["ord_alpha"]))
    err = np.min(np.abs(cosang[:, None] - targets[None, :]), axis=1)
    assert len(d) > 300 and np.max(err) < 1e-12
    both = [np.count_nonzero(np.abs(cosang - x) < 1e-9) for x in targets]
    assert min(both) > 50, both


def test_rate_quadrature_matches_cone_integral():
    s = flat()
    c = ob.ray_constants(s, 8.0)
    a0 = c["alpha_B"]
    for a in (a0, a0 + 0.02, a0 - 0.1, a0 + 0.3):
        expect = cone_rate(c["Q"], a0, a, lambda t: gauss_W(t, 0.35), far=False)
        assert ob.reflection_rate(s, 8.0, a) == pytest.approx(expect, rel=2e-7)


def test_vmf_rate_closed_form():
    # W = exp((cos theta - 1) / s^2): along the cone cos theta = S + C cos psi, and
    # int_0^2pi exp(C cos psi / s^2) dpsi = 2 pi I0(C / s^2); int W dOmega = 2 pi s^2 (1 - exp(-2 / s^2))
    fwhm = 0.05
    sg = fwhm / (2 * math.sqrt(2 * LN2))
    s = flat(mdf="vmf", mdf_fwhm_rad=fwhm)
    c = ob.ray_constants(s, 8.0)
    a0 = c["alpha_B"]
    x = 1.0 / sg ** 2
    Z = sg ** 2 * (1 - math.exp(-2 * x))
    G = 0.5 * (1 + math.cos(2 * a0) ** 2)
    for a in (a0, a0 + 0.01, a0 - 0.04):
        S, C = math.sin(a) * math.sin(a0), math.cos(a) * math.cos(a0)
        near = math.exp((S + C - 1) * x) * special.i0e(C * x) / Z
        assert ob.reflection_rate(s, 8.0, a) == pytest.approx(c["Q"] * math.cos(a0) * G * near, rel=1e-7)


def test_candidate_rate_bound():
    # majorant: mu0 + Q cos a~0 * 2 cones * 2 pi f(0), f(0) = W(0) / int W dOmega
    s = flat()
    c = ob.ray_constants(s, 8.0)
    Z = integrate.quad(lambda t: gauss_W(t, 0.35) * math.sin(t), 0.0, math.pi, epsabs=0, epsrel=1e-12)[0]
    bound = c["Q"] * math.cos(c["alpha_B"]) * 2.0 / Z
    assert c["mubar"] == pytest.approx(c["mu0"] + bound, rel=1e-9)
    shifted = ob.ray_constants(dict(s, irc_shift_rad=2e-3), 8.0)
    assert shifted["ord_qr"][0] == pytest.approx(c["Q"] * math.cos(c["alpha_B"] + 2e-3) * 2.0 / Z, rel=1e-9)


@pytest.mark.parametrize("sampler", ["thinned", "plain"])
@pytest.mark.parametrize("offset", [0.0, 0.05])
def test_thin_slab_reflection_probability(offset, sampler):
    s = flat(sampler=sampler)
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + offset
    r = cone_rate(c["Q"], c["alpha_B"], a, lambda t: gauss_W(t, 0.35))
    p = slab_probability(r, c["mu0"], 0.002 / math.sin(a))
    n = 400_000
    _, t, _ = ob.trace(s, pencil(a), n, seed=11 + int(offset * 100))
    got = n - t["refl_hist"][0]
    assert abs(got - n * p) < 4.5 * math.sqrt(n * p * (1 - p)), (got, n * p)
    assert got > 5000


@pytest.mark.parametrize("mdf,W", [("gaussian", lambda t: gauss_W(t, 0.02)),
                                   ("lorentzian", lambda t: 1.0 / (1.0 + 4.0 * t ** 2 / 0.02 ** 2))])
@pytest.mark.parametrize("offset", [0.0, 0.004])
def test_thin_slab_probability_narrow_mosaic_window(mdf, W, offset):
    # a 0.02 rad mosaic: on the facing cone the MDF exceeds v* W(0) only in a window of
    # a few hundredths of a radian of psi, so nearly all of the thinned bound sits in
    # the window and the rest of the cone carries the v* bound; the walk's first-
    # reflection probability must still follow the cone quadrature
    s = flat(mdf=mdf, mdf_fwhm_rad=0.02, sampler="thinned", refl_K_per_mm2=4e9)
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + offset
    r = cone_rate(c["Q"], c["alpha_B"], a, W)
    p = slab_probability(r, c["mu0"], 0.002 / math.sin(a))
    n = 400_000
    _, t, _ = ob.trace(s, pencil(a), n, seed=41 + int(offset * 1000))
    got = n - t["refl_hist"][0]
    assert abs(got - n * p) < 4.5 * math.sqrt(n * p * (1 - p)), (got, n * p)
    assert got > 2000
    # and it draws far fewer candidates than the plain sampler (bound 2 pi f(0) on both cones)
    _, tp, _ = ob.trace(dict(s, sampler="plain"), pencil(a), 20_000, seed=43)
    assert t["collisions"] / n < 0.1 * tp["collisions"] / 20_000


def test_limit_of_narrow_box_curves():
    s = flat()
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + 0.05
    n = 300_000
    _, tn, _ = ob.trace(s, pencil(a), n, seed=21)
    pn = (n - tn["refl_hist"][0]) / n
    # a box curve of unit area and width w -> delta as w -> 0 (the rate changes by O(w^2))
    box = dict(s, irc="box", irc_fwhm_rad=1e-6, sampler="thinned")
    _, tb, _ = ob.trace(box, pencil(a), n, seed=22)
    pb = (n - tb["refl_hist"][0]) / n
    sd = math.sqrt(pn * (1 - pn) / n + pb * (1 - pb) / n)
    assert abs(pn - pb) < 4.5 * sd, (pn, pb)


def test_two_polarisations_reflect_twice_the_unpolarised():
    # G(p1) + G(p2) = 2 - (1 - (k.k_s)^2) = 1 + cos^2 2a = 2 G_unpol for p1, p2, k orthonormal
    s = flat()
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + 0.02
    n = 300_000
    got = []
    for seed, pol in ((31, None), (32, [0.0, 1.0, 0.0]), (33, [math.sin(a), 0.0, math.cos(a)])):
        _, t, _ = ob.trace(s, pencil(a, pol=pol), n, seed=seed)
        got.append(n - t["refl_hist"][0])
    u, p1, p2 = got
    # thin slab: counts are nearly linear in G; compare p1 + p2 with 2 u
    sd = math.sqrt(p1 + p2 + 4 * u)
    assert abs(p1 + p2 - 2 * u) < 4.5 * sd + 0.02 * u, got
    # sigma polarisation (p perpendicular to the scattering plane) reflects more: G = 1 against cos^2 2a~0 = 0.79
    # for crystallites in the plane; the 0.35 rad mosaic tilts many out of it
    assert p1 > 1.1 * p2


@pytest.mark.parametrize("name,mdf", [("von_hamos_hapg", "pseudo_voigt"), ("flat_hopg_mono", "gaussian"),
                                      ("von_hamos_hapg", "lorentzian"), ("flat_hopg_mono", "uniform")])
def test_thinned_cone_bound_agrees_with_plain(name, mdf):
    w = getattr(W, name)()
    s = dict(w["spec"], irc="none", mdf=mdf, refl_K_per_mm2=2e9)
    if mdf == "uniform":
        s["mdf_fwhm_rad"] = 0.02
    n = 200_000
    _, tp, rp = ob.trace(dict(s, sampler="plain"), w["source"], n, 7, records=True)
    _, tt, rt = ob.trace(dict(s, sampler="thinned"), w["source"], n, 8, records=True)
    for key in ("absorbed", "exit_front", "exit_back", "det_hits"):
        a, b = tp[key], tt[key]
        assert abs(a - b) < 4.5 * math.sqrt(a + b + 1), (key, a, b)
    for h in range(1, 4):
        a, b = tp["refl_hist"][h], tt["refl_hist"][h]
        assert abs(a - b) < 4.5 * math.sqrt(a + b + 1), (h, a, b)
    assert tt["exit_front"] > 300
    assert tt["collisions"] < tp["collisions"] / 4
    # where the reflected rays land: the dispersive coordinate's mean and spread
    ua, ub = rp["u_mm"][rp["det_hit"] == 1], rt["u_mm"][rt["det_hit"] == 1]
    se = math.sqrt(ua.var() / len(ua) + ub.var() / len(ub))
    assert abs(ua.mean() - ub.mean()) < 4.5 * se


def test_conservation_and_thread_invariance():
    w = W.von_hamos_hapg()
    s = dict(w["spec"], irc="none", mdf="gaussian", mdf_fwhm_rad=0.05)
    img1, t1, _ = ob.trace(s, w["source"], 20_000, 9, n_threads=1)
    img4, t4, _ = ob.trace(s, w["source"], 20_000, 9, n_threads=4)
    assert t1 == t4 and np.array_equal(img1, img4)
    out = sum(t1[k] for k in ("miss", "absorbed", "exit_front", "exit_back", "exit_side", "capped", "stuck"))
    assert out == t1["emitted"] == 20_000
    assert t1["det_hits"] <= t1["exit_front"] + t1["exit_back"] + t1["exit_side"]
    assert t1["det_hits"] > 0


def test_crystallite_sampler_refuses_none():
    with pytest.raises(RuntimeError):
        ob.sample_crystallites(flat(), 8.0, 0.25, 10, 1)
