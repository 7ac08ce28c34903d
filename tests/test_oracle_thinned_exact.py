"""Exactness of the thinned candidate sampler, checked directly on its bounds.

The thinned walk never draws, per straight segment, the scatter candidates
whose marks put them outside (a) v < v* and (b) [tilt q in [qmin, 2 - qmin],
azimuth in the arcs where |k.n| lies in the window (S1, S2) of |Delta| < X*].
The sampler is exact if and only if none of the candidates it drops could
reflect, and stream (b) is drawn at a rate no smaller than the true one.  Each
of these conditions is checked here with geometry written in numpy, on random
straight segments of flat and cylindrical crystals (entering and reflected
directions, near and far from the Bragg angle), for every mosaic distribution
and rocking curve, several reflection orders and an energy-dependent rocking
curve; the oracle supplies only the bounds it computed for each segment and
its (separately pinned) curves R and W:

  * the rocking curve: R(x) / R_max <= v* for every |x| >= X* (X* is where
    the acceptance test becomes impossible for v >= v*);
  * the tilt bound: every crystallite tilted by q < qmin (or q > 2 - qmin)
    has |Delta| >= X* at every point of the segment and every azimuth, so with
    G <= 1 it cannot pass v < R G / R_max with v >= v*;
  * the table-word start of stream (b): every word below w0 maps to a tilt
    below qmin, so no word whose tilt can reflect is left out of (b);
  * the arc bound: the measure P_xi of azimuths in the window is at most pbar
    for every tilt in [qmin, 2 - qmin] at every point of the segment;
  * band B of stream (b) (one reflection order): its table words [w1, w2) map
    to tilts in [qmin, q_J] beyond the band's first knot, where P_xi is at most
    pbarB < pbar at every point of the segment; the words of band A and band B
    together are exactly [w0, 2^32), and band A's share is its rate's share;
  * no rocking curve (candidates on the Bragg cones): W / W(0) on the cone
    facing the ray is at most wn everywhere, at most v* outside |psi| < psis,
    and at most wf on the other cone.
"""
import math

import numpy as np
import pytest

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

DEG = math.pi / 180.0
MDFS = [("gaussian", {}), ("lorentzian", {}), ("pseudo_voigt", {"mdf_eta": 0.5}), ("vmf", {}), ("wl", {}),
        ("swl", {}), ("uniform", {})]
IRCS = [("darwin", {}), ("darwin_prins", {"prins_g": 0.05}), ("pseudo_voigt", {"irc_lorentz_fwhm_rad": 8e-6}),
        ("gaussian", {}), ("lorentzian", {}), ("box", {})]


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _frame(spec):
    a = np.array(spec["axis"], float)
    if spec["geometry"] == "flat":
        N = _unit(np.array(spec["normal"], float))
        ed = _unit(a - a.dot(N) * N)
        return N, ed, np.cross(N, ed)
    ax = _unit(a)
    cc = np.array(spec["normal"], float)
    cc = _unit(cc - cc.dot(ax) * ax)
    return ax, cc, np.cross(ax, cc)


def local_normal(spec, x):
    """unit crystal normal at points x (n, 3): flat: N; cylinder: toward the axis"""
    if spec["geometry"] == "flat":
        N, _, _ = _frame(spec)
        return np.broadcast_to(N, x.shape).copy()
    ax, _, _ = _frame(spec)
    rel = x - np.array(spec["centre_mm"], float)
    radial = rel - (rel @ ax)[:, None] * ax
    return -_unit(radial)


def random_segments(spec, rng, n, alpha0, spread=0.03):
    """points in the crystal and directions about the Bragg angle alpha0:
    entering (k.N < 0) and leaving the front face (k.N > 0, as after a
    reflection), most within +-spread of alpha0, some far off it"""
    t = spec["thickness_mm"]
    depth = np.where(rng.random(n) < 0.5, 0.0, rng.random(n) * t)
    u = (rng.random(n) - 0.5) * 0.9 * spec["size_disp_mm"]
    v = (rng.random(n) - 0.5) * 0.9 * spec["size_nondisp_mm"]
    if spec["geometry"] == "flat":
        N, ed, en = _frame(spec)
        c = np.array(spec["centre_mm"], float)
        x = c + u[:, None] * ed + v[:, None] * en - depth[:, None] * N
        Nx = np.broadcast_to(N, x.shape)
        t1 = np.broadcast_to(ed, x.shape)
    else:
        ax, cc, ww = _frame(spec)
        R = spec["radius_mm"]
        phi = v / R
        r = R + depth
        c = np.array(spec["centre_mm"], float)
        x = (c + (spec["centre_axial_mm"] + u)[:, None] * ax + (r * np.cos(phi))[:, None] * cc +
             (r * np.sin(phi))[:, None] * ww)
        Nx = local_normal(spec, x)
        t1 = np.broadcast_to(ax, x.shape)
    t2 = np.cross(Nx, t1)
    dalpha = np.where(rng.random(n) < 0.8, (rng.random(n) - 0.5) * 2 * spread, (rng.random(n) - 0.5) * 0.6)
    alpha = np.clip(alpha0 + dalpha, 1e-3, 0.5 * math.pi - 1e-3)
    az = np.where(rng.random(n) < 0.7, (rng.random(n) - 0.5) * 0.2, rng.random(n) * 2 * math.pi)
    up = np.where(rng.random(n) < 0.3, 1.0, -1.0)
    k = (np.cos(alpha) * np.cos(az))[:, None] * t1 + (np.cos(alpha) * np.sin(az))[:, None] * t2 + \
        (up * np.sin(alpha))[:, None] * Nx
    return x, _unit(k)


def _points(spec, x, k, s_exit, m=9):
    """m points along each segment (n, m, 3) and the normal there"""
    f = np.linspace(0.0, 1.0, m)
    P = x[:, None, :] + (s_exit[:, None] * f)[:, :, None] * k[:, None, :]
    N = local_normal(spec, P.reshape(-1, 3)).reshape(P.shape)
    return P, N


def _kn_range(kN, kt, q):
    """range of |k.n| over the azimuths of a crystallite tilted by q from N"""
    b = np.sqrt(q * (2.0 - q)) * kt
    lo, hi = kN * (1.0 - q) - b, kN * (1.0 - q) + b
    amin = np.where((lo <= 0) & (hi >= 0), 0.0, np.minimum(np.abs(lo), np.abs(hi)))
    amax = np.maximum(np.abs(lo), np.abs(hi))
    return np.clip(amin, 0, 1), np.clip(amax, 0, 1)


def _arc_measure(a, b, S1, S2):
    """measure (in units of pi) of xi' in [0, pi] with |a + b cos xi'| in (S1, S2)"""
    tot = np.zeros(np.broadcast(a, b, S1, S2).shape)
    for lo, hi in (((S1 - a) / b, (S2 - a) / b), ((-S2 - a) / b, (-S1 - a) / b)):
        l, h = np.clip(lo, -1, 1), np.clip(hi, -1, 1)
        tot += np.where(l < h, np.arccos(l) - np.arccos(h), 0.0)
    return tot / math.pi


_TABLES = {}


def _table(spec):
    key = repr(sorted(spec.items()))
    if key not in _TABLES:
        _TABLES[key] = ob.mdf_table(spec)
    return _TABLES[key]


def check_segments(spec, E, x, k, order=0, width=1.0):
    """all exactness conditions on the segments (x, k) at energies E; returns
    the number of segments where the thinned bounds were in force"""
    B = ob.segment_bounds(spec, E, x, k, order)
    act = (B["thinned"] == 1) & (B["ra"] < 1.0)
    if not act.any():
        return 0
    xs, ks = x[act], k[act]
    a0, xstar, vstar = B["alpha0"][act], B["xstar"][act], B["vstar"][act]
    qmin, pbar, S1, S2 = B["qmin"][act], B["pbar"][act], B["S1"][act], B["S2"][act]
    s_exit = np.minimum(B["s_exit"][act], 1e3)
    # the rocking curve beyond X* (this order's width scale)
    rmax = B["irc_max"][0]
    xs_ = np.unique(xstar)
    for X in (xs_.min(), xs_.max()):
        grid = X * np.geomspace(1.0, 1e4, 120)
        r = ob.irc(spec, grid / width) / rmax
        r2 = ob.irc(spec, -grid / width) / rmax
        assert np.all(r <= vstar[0] * (1 + 1e-9)) and np.all(r2 <= vstar[0] * (1 + 1e-9)), X
    # the window is that of |Delta| < X*
    assert np.allclose(S1, np.sin(np.maximum(0, a0 - xstar)), rtol=0, atol=1e-15)
    assert np.allclose(S2, np.sin(np.minimum(0.5 * math.pi, a0 + xstar)), rtol=0, atol=1e-15)
    # tilt bound at every point of the segment
    P, N = _points(spec, xs, ks, s_exit)
    kN = np.einsum("nmi,ni->nm", N, ks)
    kt = np.sqrt(np.clip(1.0 - kN * kN, 0.0, 1.0))
    for q in (qmin, 2.0 - qmin):
        mn, mx = _kn_range(kN, kt, q[:, None])
        dist = np.maximum(a0[:, None] - np.arcsin(mx), np.arcsin(mn) - a0[:, None])
        assert np.all(dist >= xstar[:, None] * (1 - 1e-9)), float((dist / xstar[:, None]).min())
    # stream (b) starts at a word whose tilt is below qmin
    tab = _table(spec)
    w0 = B["w0"][act]
    for w, qm in zip(w0, qmin):
        if w > 0:
            assert ob.mdf_table_lookup(tab, [int(w) - 1])[0] < qm
    # arc bound: P_xi <= pbar for tilts in [qmin, 2 - qmin] everywhere on the segment
    th0 = 2.0 * np.arcsin(np.sqrt(0.5 * qmin))
    # the largest arc measure sits just above the smallest tilt (the window near the edge of
    # the azimuth range): resolved finely there, coarsely beyond
    frac = np.concatenate([1.0 + np.geomspace(1e-7, 0.05, 160), np.geomspace(1.05, 50.0, 60)])
    for f in frac:
        th = np.minimum(th0 * f, math.pi - th0)
        q = (2.0 * np.sin(0.5 * th) ** 2)[:, None]
        b = np.sqrt(q * (2.0 - q)) * kt
        a = kN * (1.0 - q)
        pxi = _arc_measure(a, np.maximum(b, 1e-300), S1[:, None], S2[:, None])
        assert np.all(pxi <= pbar[:, None] * (1 + 1e-9) + 1e-15), float((pxi / pbar[:, None]).max())
    check_band_b(spec, B, act, tab, kN, kt, S1, S2)
    return int(act.sum())


QJ = 2.0 ** (351 / 8.0 - 48.0)       # band B's largest tilt, q_J = 2^(-33/8)


def check_band_b(spec, B, act, tab, kN, kt, S1, S2):
    """band B of stream (b): words, tilts and the arc bound pbarB"""
    w0, w1, w2 = B["w0"][act], B["w1"][act], B["w2"][act]
    pbar, pbarB, sA, qmin = B["pbar"][act], B["pbarB"][act], B["sA"][act], B["qmin"][act]
    on = w1 < w2
    assert np.all(w0 <= w1) and np.all(w1 <= w2)
    assert np.all(~on | (pbarB < pbar)) and np.all(on | ((w1 == w0) & (w2 == w0) & (sA == 1.0)))
    # band A's share of stream (b) is that of its rate (words x bound)
    spanA = (w1 - w0).astype(np.float64) + (2.0 ** 32 - w2.astype(np.float64))
    lA, lB = spanA * pbar, (w2 - w1).astype(np.float64) * pbarB
    assert np.allclose(sA[on], (lA / (lA + lB))[on], rtol=1e-12, atol=0)
    for i in np.flatnonzero(on):
        # the band's tilts: beyond qmin, from the knot that starts w1's interval, at most q_J
        qlo, qhi = ob.mdf_table_lookup(tab, [int(w1[i]), int(w2[i]) - 1])
        assert qlo >= qmin[i] and qhi <= QJ * (1 + 1e-12), (qlo, qhi, qmin[i])
        # P_xi <= pbarB over the band's tilts everywhere on the segment (fine near its first tilt)
        t_lo, t_hi = 2.0 * math.asin(math.sqrt(0.5 * qlo)), 2.0 * math.asin(math.sqrt(0.5 * QJ))
        th = np.concatenate([t_lo * (1.0 + np.geomspace(1e-9, 0.1, 60)), np.linspace(t_lo, t_hi, 120)])
        q = (2.0 * np.sin(0.5 * th) ** 2)[:, None]
        b = np.sqrt(q * (2.0 - q)) * kt[i][None, :]
        pxi = _arc_measure(kN[i][None, :] * (1.0 - q), np.maximum(b, 1e-300), S1[i], S2[i])
        assert np.all(pxi <= pbarB[i] * (1 + 1e-9) + 1e-15), (float(pxi.max()), float(pbarB[i]))
    return int(on.sum())


def _spec(geometry, mdf, mdf_kw, irc, irc_kw, fwhm_deg=0.2, **extra):
    if geometry == "flat":
        s = dict(W.flat_hopg_mono()["spec"])
    else:
        s = dict(W.von_hamos_hapg()["spec"])
    s.update(mdf=mdf, mdf_fwhm_rad=fwhm_deg * DEG, irc=irc, irc_fwhm_rad=20e-6, mdf_eta=0.0, prins_g=0.0,
             irc_lorentz_fwhm_rad=0.0, sampler="thinned")
    s.update(mdf_kw)
    s.update(irc_kw)
    s.update(extra)
    return s


@pytest.mark.parametrize("geometry,mdf,mdf_kw", [("cyl", m, kw) for m, kw in MDFS] +
                         [("flat", "gaussian", {})])
def test_thinned_bounds_drop_nothing_that_can_reflect_every_mdf(geometry, mdf, mdf_kw):
    rng = np.random.default_rng(hash((geometry, mdf)) % 2**32)
    s = _spec(geometry, mdf, mdf_kw, "darwin_prins", {"prins_g": 0.05}, fwhm_deg=0.1 if mdf != "uniform" else 0.4)
    a0 = ob.ray_constants(s, 8.0)["alpha_B"]
    x, k = random_segments(s, rng, 400, a0)
    E = 8.0 + (rng.random(len(x)) - 0.5) * 0.2
    assert check_segments(s, E, x, k) > 100


@pytest.mark.parametrize("geometry,irc,irc_kw", [("flat", r, kw) for r, kw in IRCS] +
                         [("cyl", r, kw) for r, kw in IRCS[:2]])
def test_thinned_bounds_drop_nothing_that_can_reflect_every_rocking_curve(geometry, irc, irc_kw):
    rng = np.random.default_rng(hash((geometry, irc)) % 2**32)
    s = _spec(geometry, "gaussian", {}, irc, irc_kw, fwhm_deg=0.3)
    a0 = ob.ray_constants(s, 8.0)["alpha_B"]
    x, k = random_segments(s, rng, 400, a0)
    E = np.full(len(x), 8.0)
    assert check_segments(s, E, x, k) > 100


def test_thinned_bounds_several_orders_and_energy_table():
    # graphite (002), (004), (006) with a wider second and third order, and a rocking
    # curve that widens and shifts with energy: each order's bounds on its own X*
    rng = np.random.default_rng(11)
    s = _spec("cyl", "gaussian", {}, "pseudo_voigt", {"irc_lorentz_fwhm_rad": 8e-6}, fwhm_deg=0.2,
              orders=[(1, 1.0, 1.0), (2, 0.6, 1.5), (3, 0.3, 2.0)],
              irc_energy=[(7.5, 0.8, -5e-6), (8.5, 1.3, 5e-6)])
    n_act = 0
    for h in range(3):
        rc = ob.ray_constants(s, 8.0)
        a0 = rc["ord_alpha"][h]
        x, k = random_segments(s, rng, 300, a0)
        # the order's width at each energy: the table's scale times the order's ratio
        for Ei in (7.7, 8.0, 8.3):
            w = ob.ray_constants(s, Ei)["ord_w"][h]
            n_act += check_segments(s, np.full(len(x), Ei), x, k, order=h, width=w)
    assert n_act > 300


def test_thinned_bounds_small_vstar_and_narrow_mosaic():
    rng = np.random.default_rng(5)
    for vs, fw in ((2.0 ** -10, 0.05), (2.0 ** -2, 0.5)):
        s = _spec("flat", "vmf", {}, "lorentzian", {}, fwhm_deg=fw, thin_vstar=vs)
        a0 = ob.ray_constants(s, 8.0)["alpha_B"]
        x, k = random_segments(s, rng, 300, a0, spread=0.01)
        assert check_segments(s, np.full(len(x), 8.0), x, k) > 50


def _cone_check(spec, E, x, k):
    B = ob.segment_bounds(spec, E, x, k, 0)
    act = B["thinned"] == 1
    xs, ks = x[act], k[act]
    W0 = B["W0"][0]
    vstar = B["vstar"][0]
    P, N = _points(spec, xs, ks, np.minimum(B["s_exit"][act], 1e3), m=5)
    psi = np.linspace(-math.pi, math.pi, 241)
    for i in range(len(xs)):
        a0 = B["alpha0"][act][i]
        s0, c0 = math.sin(a0), math.cos(a0)
        for j in range(P.shape[1]):
            Nj = N[i, j]
            kk = ks[i]
            kN = float(kk @ Nj)
            e1 = Nj - kN * kk
            if np.linalg.norm(e1) < 1e-12:
                continue
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(kk, e1)
            side = -1.0 if kN < 0 else 1.0
            for sg, bound, outside in ((side, B["wn"][act][i], True), (-side, B["wf"][act][i], False)):
                n = sg * s0 * kk + c0 * (np.cos(psi)[:, None] * e1 + np.sin(psi)[:, None] * e2)
                q = np.clip(1.0 - n @ Nj, 0.0, 2.0)
                Wr = ob.mdf_W(spec, q) / W0
                assert np.all(Wr <= bound * (1 + 1e-9) + 1e-15), (sg, float(Wr.max()), bound)
                if outside:
                    out = np.abs(psi) >= B["psis"][act][i]
                    assert np.all(Wr[out] <= vstar * (1 + 1e-9) + 1e-15), float(Wr[out].max(initial=0))
    return int(act.sum())


@pytest.mark.parametrize("geometry,mdf,fw", [("cyl", "gaussian", 0.4), ("flat", "gaussian", 0.2),
                                             ("cyl", "vmf", 1.0), ("flat", "wl", 0.3), ("cyl", "swl", 0.3),
                                             ("flat", "pseudo_voigt", 0.2)])
def test_cone_bounds_without_rocking_curve(geometry, mdf, fw):
    rng = np.random.default_rng(hash((geometry, mdf, "none")) % 2**32)
    s = _spec(geometry, mdf, {"mdf_eta": 0.5} if mdf == "pseudo_voigt" else {}, "none", {}, fwhm_deg=fw)
    a0 = ob.ray_constants(s, 8.0)["alpha_B"]
    x, k = random_segments(s, rng, 12, a0, spread=0.02)
    assert _cone_check(s, np.full(len(x), 8.0), x, k) > 6


def test_thinned_bounds_long_chords_in_a_thick_cylinder():
    # rays entering a thick shell at a few degrees and travelling around it on long
    # chords: |k.N| changes along the segment, so the bounds must hold over its whole range
    rng = np.random.default_rng(21)
    s = _spec("cyl", "gaussian", {}, "darwin", {}, fwhm_deg=0.5, thickness_mm=2.0)
    a0 = ob.ray_constants(s, 8.0)["alpha_B"]
    x, k = random_segments(s, rng, 600, a0, spread=0.2)
    B = ob.segment_bounds(s, np.full(len(x), 8.0), x, k, 0)
    assert np.max(np.abs(np.abs(B["kN1"]) - np.abs(B["kN0"]))) > 0.05
    assert check_segments(s, np.full(len(x), 8.0), x, k) > 100
