"""Pins of higher-order reflections (the cross-section summed over the
reflections H, Sec. 2.2.3) and of the energy-dependent rocking curve (its width
and peak shift as functions of energy, Sec. 2.1).

* an explicit first order only is the single reflection, word for word;
* order m on planes d equals order 1 on planes d / m (Bragg's law on d / m);
* the per-order constants follow Bragg's law and the definition of Q;
* the first-reflection probability of a thin slab equals the quadrature of
  Eq. (ReflXsection) summed over the orders, and the share of each order
  (told apart by the scattering angle) equals its share of the quadrature;
* a constant energy table is the same spectrometer with a wider, shifted
  rocking curve; the table interpolates linearly and clamps at its ends;
* the thinned and plain samplers agree with two orders."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W


def flat(**kw):
    s = dict(W.flat_hopg_mono()["spec"], refl_K_per_mm2=5.5e8)   # ~ the Darwin-width value at 8 keV
    s.update(kw)
    return s


def pencil(alpha, E=8.0, dist=300.0):
    ca, sa = math.cos(alpha), math.sin(alpha)
    return dict(components=[dict(kind="mono", e0_keV=E, weight=1.0)],
                origin_mm=[-dist * ca, 0.0, dist * sa], axis=[ca, 0.0, -sa],
                cone_half_angle_rad=0.0, spot_fwhm_mm=(0.0, 0.0))


@pytest.mark.parametrize("sampler", ["plain", "thinned"])
def test_explicit_first_order_is_the_single_reflection(sampler):
    w = W.flat_hopg_mono()
    s0 = dict(w["spec"], sampler=sampler)
    s1 = dict(s0, orders=[(1, 1.0, 1.0)])
    _, t0, r0 = ob.trace(s0, w["source"], 20_000, 3, records=True)
    _, t1, r1 = ob.trace(s1, w["source"], 20_000, 3, records=True)
    assert t0 == t1
    for f in ("outcome", "nrefl", "ncoll", "ix", "iy"):
        assert np.array_equal(r0[f], r1[f]), f
    assert np.array_equal(r0["pos"], r1["pos"])


def test_order_m_on_d_is_order_one_on_d_over_m():
    s = flat(d_spacing_A=3.354)
    half = dict(s, d_spacing_A=3.354 / 2)
    s2 = dict(s, orders=[(2, 1.0, 1.0)])
    E = 9.0
    a2 = ob.ray_constants(half, E)["alpha_B"]
    src = pencil(a2 + 2e-4, E=E)
    _, ta, ra = ob.trace(half, src, 20_000, 5, records=True)
    _, tb, rb = ob.trace(s2, src, 20_000, 5, records=True)
    assert ta == tb
    assert np.array_equal(ra["nrefl"], rb["nrefl"]) and np.array_equal(ra["ncoll"], rb["ncoll"])
    assert np.allclose(ra["pos"], rb["pos"], rtol=0, atol=1e-12)
    assert ta["exit_front"] > 100


def test_per_order_constants():
    s = flat(orders=[(1, 1.0, 1.0), (2, 0.5, 0.4), (3, 0.2, 0.3)])
    E = 12.0
    c = ob.ray_constants(s, E)
    c1 = ob.ray_constants(flat(), E)
    lam = 12.398419843320026 / E
    for h, m in enumerate((1, 2, 3)):
        assert c["ord_sin"][h] == pytest.approx(m * lam / (2 * 3.354), rel=1e-15)
    # Q_h = (K_rel K)^2 lambda^3 / sin(2 a_h): relative to the first order
    for h, (kr, _) in enumerate(((1.0, 1.0), (0.5, 0.4), (0.2, 0.3))):
        a = c["ord_alpha"][h]
        expect = c1["Q"] * kr ** 2 * math.sin(2 * c["ord_alpha"][0]) / math.sin(2 * a)
        assert c["ord_Q"][h] == pytest.approx(expect, rel=1e-12)
    # the majorant: mu0 + sum_h Q_h R_max / w_h, R_max of the described curve
    rmax = ob.irc_max(s)
    assert c["mubar"] == pytest.approx(c["mu0"] + sum(q * rmax / w for q, w in zip(c["ord_Q"], (1.0, 0.4, 0.3))),
                                       rel=1e-14)
    # an order without a Bragg solution drops out
    low = ob.ray_constants(s, 2.5)
    assert math.isnan(low["ord_alpha"][1]) and low["ord_qr"][1] == 0 and not low["no_bragg"]
    assert ob.ray_constants(s, 1.5)["no_bragg"]


def test_two_order_reflection_probability_and_shares_match_quadrature():
    # a Gaussian mosaic 0.35 rad wide: a pencil at 0.36 rad meets crystallites at
    # both Bragg angles (0.232 and 0.483 rad at 8 keV); thin strongly reflecting
    # slab, one reflection
    s = flat(mdf="gaussian", mdf_fwhm_rad=0.35, thickness_mm=0.002, max_reflections=1, irc="gaussian",
             irc_fwhm_rad=2e-3, orders=[(1, 1.0, 1.0), (2, 0.6, 1.5)], sampler="plain", refl_K_per_mm2=1.5e10)
    a = 0.36
    r = ob.reflection_rate(s, 8.0, a)
    r1 = ob.reflection_rate(dict(s, orders=[(1, 1.0, 1.0)]), 8.0, a)
    r2 = ob.reflection_rate(dict(s, orders=[(2, 0.6, 1.5)]), 8.0, a)
    assert r == pytest.approx(r1 + r2, rel=1e-9)
    c = ob.ray_constants(s, 8.0)
    L = 0.002 / math.sin(a)
    mu = c["mu0"]
    p = r / (r + mu) * (1 - math.exp(-(r + mu) * L))
    n = 400_000
    _, t, rec = ob.trace(s, pencil(a), n, seed=9, records=True)
    got = n - t["refl_hist"][0]
    sd = math.sqrt(n * p * (1 - p))
    assert abs(got - n * p) < 4.5 * sd, (got, n * p)
    # the order of each reflection from its scattering angle 2 a~ (near 2 a_B of the order)
    refl = rec["nrefl"] == 1
    k0 = np.array([math.cos(a), 0.0, -math.sin(a)])
    scat = np.arccos(np.clip(rec["dir"][refl] @ k0, -1, 1))
    two = np.count_nonzero(scat > c["ord_alpha"][0] + c["ord_alpha"][1])
    frac = r2 / r
    m = int(refl.sum())
    assert abs(two - m * frac) < 4.5 * math.sqrt(m * frac * (1 - frac)), (two, m * frac)
    assert 0.1 < frac < 0.9


def test_constant_energy_table_is_a_wider_shifted_curve():
    w = W.flat_hopg_mono()
    base = dict(w["spec"], refl_K_per_mm2=5.5e8, irc="darwin", irc_fwhm_rad=20e-6)
    tab = dict(base, irc_energy=[(8.0, 2.0, 3e-5)])
    wide = dict(base, irc_fwhm_rad=40e-6, irc_shift_rad=3e-5)
    for sampler in ("plain", "thinned"):
        _, ta, ra = ob.trace(dict(tab, sampler=sampler), w["source"], 30_000, 8, records=True)
        _, tb, rb = ob.trace(dict(wide, sampler=sampler), w["source"], 30_000, 8, records=True)
        assert ta["exit_front"] > 200
        same = (ra["outcome"] == rb["outcome"]) & (ra["nrefl"] == rb["nrefl"])
        assert same.mean() > 0.9999
        assert np.allclose(ra["pos"][same], rb["pos"][same], rtol=0, atol=1e-9)


def test_energy_table_interpolates_and_clamps():
    knots = [(7.0, 1.0, 0.0), (8.0, 2.0, 1e-5), (9.0, 1.5, -2e-5)]
    s = flat(irc_energy=knots, irc_shift_rad=5e-6, orders=[(1, 1.0, 1.0), (2, 0.5, 0.5)])
    xs, ws, ss = zip(*knots)
    for E in (6.0, 7.0, 7.25, 8.0, 8.6, 9.0, 11.0):
        c = ob.ray_constants(s, E)
        assert c["ord_w"][0] == pytest.approx(np.interp(E, xs, ws), rel=1e-14)
        assert c["ord_w"][1] == pytest.approx(0.5 * np.interp(E, xs, ws), rel=1e-14)
        assert c["shift_rad"] == pytest.approx(5e-6 + np.interp(E, xs, ss), rel=1e-12, abs=1e-20)


def test_two_orders_thinned_agrees_with_plain():
    w = W.von_hamos_hapg()
    s = dict(w["spec"], orders=[(1, 1.0, 1.0), (2, 0.5, 0.7)], irc_energy=[(7.5, 0.8, 0.0), (8.5, 1.3, 1e-5)])
    n = 300_000
    _, tp, _ = ob.trace(dict(s, sampler="plain"), w["source"], n, seed=31)
    _, tt, _ = ob.trace(dict(s, sampler="thinned"), w["source"], n, seed=32)
    for key in ("miss", "absorbed", "exit_front", "exit_back", "det_hits"):
        a, b = tp[key], tt[key]
        assert abs(a - b) < 4.5 * math.sqrt(a + b + 1), (key, a, b)
    assert tt["collisions"] < tp["collisions"] / 2


def test_invalid_orders_and_tables_rejected():
    w = W.flat_hopg_mono()
    for bad in [dict(orders=[(0, 1.0, 1.0)]), dict(orders=[(1, -1.0, 1.0)]), dict(orders=[(1, 1.0, 0.0)]),
                dict(orders=[(1, 1.0, 1.0)] * 5), dict(irc_energy=[(8.0, 0.0, 0.0)]),
                dict(irc_energy=[(8.0, 1.0, 0.0), (7.0, 1.0, 0.0)])]:
        with pytest.raises(RuntimeError):
            ob.trace(dict(w["spec"], **bad), w["source"], 10, seed=1)
