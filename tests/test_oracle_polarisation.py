"""Pins of the oracle's polarised walk (Eq. G_pol, the polarisation update of
Sec. 2.2.4) and of user-supplied rays (Sec. 2.1).

* hand-traced single rays: sigma polarisation (p perpendicular to the
  scattering plane) reflects with G = 1, pi polarisation (p in the plane) with
  G = cos^2(2a), and the unpolarised factor is their mean (Eq. G_unpol);
* the reflected polarisation is the component of p perpendicular to the
  reflected direction, renormalised: closed forms for sigma / pi, invariants
  for a tilted crystallite;
* for any two orthogonal polarisations of one ray the factors add up to twice
  the unpolarised one, so randomly polarised rays reproduce the unpolarised
  reflection statistics;
* user rays that repeat what a zero-cone, zero-spot source emits give the same
  image, tallies and records as the sampled source (the walk draws the same
  Philox words from call 2 on)."""
import math

import numpy as np
import pytest

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

TINY_STEP = 0xFFFFFFFF
LONG_STEP = 0x00000000
REJECT = 0xFFFFFFFF


def flat(**kw):
    # the plain walk: the hand-traced rays below inject its word layout
    s = dict(W.flat_hopg_mono()["spec"], sampler="plain")
    s.update(kw)
    return s


def darwin_rel(x, fwhm=20e-6):
    """Darwin curve relative to its plateau at x = Delta - Delta_M (FWHM = 3 w / sqrt 2)"""
    y = abs(x) / (fwhm * math.sqrt(2) / 3)
    if y <= 1:
        return 1.0
    return 1.0 / (y + math.sqrt(y * y - 1)) ** 2


def _one_collision(s, a, pol, v):
    """a ray at glancing angle a onto a crystallite along the surface normal
    (w2 = 0), acceptance word for v; then a long step out of the crystal"""
    c = ob.ray_constants(s, 8.0)
    pa = c["p_abs"]
    w = int((pa + v * (1 - pa)) * 2**32)
    k = [math.cos(a), 0.0, -math.sin(a)]
    return ob.walk_injected(s, 8.0, [0.0, 0.0, 0.0], k, [TINY_STEP, w, 0, 0, LONG_STEP, REJECT, 0, 0], pol=pol)


@pytest.mark.parametrize("which", ["sigma", "pi", "unpolarised"])
def test_polarisation_factor_on_a_single_collision(which):
    s = flat(mdf="uniform", mdf_fwhm_rad=1e-9)
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    a = aB + 15e-6                                   # on the Darwin plateau's shoulder
    c2 = math.cos(2 * a)
    G = {"sigma": 1.0, "pi": c2 * c2, "unpolarised": 0.5 * (1 + c2 * c2)}[which]
    pol = {"sigma": [0.0, 1.0, 0.0], "pi": [math.sin(a), 0.0, math.cos(a)], "unpolarised": None}[which]
    P = darwin_rel(a - aB) * G
    assert ob.walk_injected is not None
    assert _one_collision(s, a, pol, 0.995 * P)["nrefl"] == 1
    assert _one_collision(s, a, pol, 1.005 * P)["nrefl"] == 0


def test_sigma_pi_thresholds_differ_by_cos2_2a():
    # the three factors are 1, cos^2 2a and their mean: the decisions are
    # distinct at a v between them (a dropped or swapped G fails here)
    s = flat(mdf="uniform", mdf_fwhm_rad=1e-9)
    a = ob.ray_constants(s, 8.0)["alpha_B"]
    c2 = math.cos(2 * a)
    v = 0.5 * (c2 * c2 + 0.5 * (1 + c2 * c2))        # between pi and unpolarised
    assert _one_collision(s, a, [0.0, 1.0, 0.0], v)["nrefl"] == 1
    assert _one_collision(s, a, None, v)["nrefl"] == 1
    assert _one_collision(s, a, [math.sin(a), 0.0, math.cos(a)], v)["nrefl"] == 0


def test_reflected_polarisation_sigma_and_pi_closed_forms():
    s = flat(mdf="uniform", mdf_fwhm_rad=1e-9)
    a = ob.ray_constants(s, 8.0)["alpha_B"]
    r = _one_collision(s, a, [0.0, 1.0, 0.0], 1e-6)
    assert r["nrefl"] == 1
    assert np.allclose(r["pol"], [0.0, 1.0, 0.0], atol=1e-12)
    # pi: p = (sin a, 0, cos a) -> perpendicular to k_s = (cos a, 0, sin a) in the plane
    r = _one_collision(s, a, [math.sin(a), 0.0, math.cos(a)], 1e-6)
    assert r["nrefl"] == 1
    assert np.allclose(r["dir"], [math.cos(a), 0.0, math.sin(a)], atol=1e-6)
    assert np.allclose(r["pol"], [-math.sin(a), 0.0, math.cos(a)], atol=1e-6)
    # the input polarisation is projected perpendicular to k first
    r = _one_collision(s, a, [0.0, 0.0, 5.0], 1e-6)
    assert np.allclose(r["pol"], [-math.sin(a), 0.0, math.cos(a)], atol=1e-6)


def test_reflected_polarisation_invariants_on_tilted_crystallites():
    # a box rocking curve wider than the mosaic: every candidate is inside it
    s = flat(mdf="uniform", mdf_fwhm_rad=0.02, irc="box", irc_fwhm_rad=0.2)
    c = ob.ray_constants(s, 8.0)
    aB, pa = c["alpha_B"], c["p_abs"]
    rng = np.random.default_rng(5)
    n = 400
    a = aB + rng.uniform(-0.01, 0.01, n)
    k = np.stack([np.cos(a), np.zeros(n), -np.sin(a)], 1)
    p0 = rng.normal(size=(n, 3))
    acc = int((pa + 0.9 * (1 - pa)) * 2**32)         # v = 0.9: G = 0.79 .. 1 decides
    words = np.zeros((n, 8), dtype=np.uint64)
    words[:, 0] = TINY_STEP
    words[:, 1] = acc
    words[:, 2:4] = rng.integers(0, 2**32, size=(n, 2))
    words[:, 4] = LONG_STEP
    words[:, 5] = REJECT
    r = ob.walk_injected_n(s, np.full(n, 8.0), np.zeros((n, 3)), k, words, pol=p0)
    p, d = r["pol"], r["dir"]
    assert np.all(np.abs(np.linalg.norm(p, axis=1) - 1) < 1e-12)
    assert np.all(np.abs(np.sum(p * d, 1)) < 1e-12)
    pin = p0 - np.sum(p0 * k, 1)[:, None] * k
    pin /= np.linalg.norm(pin, axis=1)[:, None]
    refl = r["nrefl"] == 1
    assert refl.sum() > 100 and (~refl).sum() > 10
    # reflected: coplanar with the incoming p and the reflected direction, on p's side
    assert np.all(np.abs(np.linalg.det(np.stack([p[refl], pin[refl], d[refl]], 1))) < 1e-10)
    assert np.all(np.sum(p[refl] * pin[refl], 1) > 0)
    # not reflected: the projected input
    assert np.allclose(p[~refl], pin[~refl], atol=1e-12)


def test_orthogonal_polarisations_average_to_unpolarised_factor():
    # G(p1) + G(p2) = 2 G_unpol for orthogonal p1, p2 perpendicular to k, for any
    # crystallite: with a box rocking curve (R = R_max wherever the candidate
    # lands) the acceptance threshold on v, found by bisection, is G
    s = flat(mdf="uniform", mdf_fwhm_rad=0.03, irc="box", irc_fwhm_rad=0.2)
    c = ob.ray_constants(s, 8.0)
    aB, pa = c["alpha_B"], c["p_abs"]
    rng = np.random.default_rng(7)
    m = 40
    a = aB + rng.uniform(-0.01, 0.01, m)
    k = np.stack([np.cos(a), np.zeros(m), -np.sin(a)], 1)
    b = rng.normal(size=(m, 3))
    p1 = b - np.sum(b * k, 1)[:, None] * k
    p1 /= np.linalg.norm(p1, axis=1)[:, None]
    p2 = np.cross(k, p1)
    w23 = rng.integers(0, 2**32, size=(m, 2))

    def thresholds(pol):
        lo = np.full(m, int(math.ceil(pa * 2**32)), dtype=np.int64)
        hi = np.full(m, 2**32 - 1, dtype=np.int64)
        for _ in range(33):
            mid = (lo + hi) // 2
            words = np.zeros((m, 8), dtype=np.uint64)
            words[:, 0] = TINY_STEP
            words[:, 1] = mid
            words[:, 2:4] = w23
            words[:, 4] = LONG_STEP
            words[:, 5] = REJECT
            r = ob.walk_injected_n(s, np.full(m, 8.0), np.zeros((m, 3)), k, words, pol=pol)
            ok = r["nrefl"] == 1
            lo = np.where(ok, mid, lo)
            hi = np.where(ok, hi, mid)
        return ((lo + 0.5) / 2**32 - pa) / (1 - pa)

    t1, t2, tu = thresholds(p1), thresholds(p2), thresholds(None)
    quantum = 2.0**-32 / (1 - pa)                        # resolution of v on one word
    assert np.all((tu > 0.5) & (tu <= 1.0))
    assert np.allclose(t1 + t2, 2 * tu, rtol=0, atol=3 * quantum)
    # each threshold is its factor: 1 - (p . k_s)^2 and (1 + (k . k_s)^2) / 2,
    # with k_s the direction an accepted walk leaves along
    words = np.zeros((m, 8), dtype=np.uint64)
    words[:, 0] = TINY_STEP
    words[:, 1] = int(math.ceil(pa * 2**32)) + 64
    words[:, 2:4] = w23
    words[:, 4] = LONG_STEP
    words[:, 5] = REJECT
    ks = ob.walk_injected_n(s, np.full(m, 8.0), np.zeros((m, 3)), k, words)["dir"]
    assert np.allclose(t1, 1 - np.sum(p1 * ks, 1) ** 2, rtol=0, atol=3 * quantum)
    assert np.allclose(tu, 0.5 * (1 + np.sum(k * ks, 1) ** 2), rtol=0, atol=3 * quantum)
    # the pair is not trivially equal to the unpolarised factor
    assert np.sum(np.abs(t1 - tu) > 1e-4) >= 30


def test_random_polarisation_user_rays_reproduce_unpolarised_statistics():
    w = W.flat_hopg_mono()
    s = w["spec"]
    rays = _rays_of_source(w["source"], 100_000, seed=3)
    n = len(rays["E"])
    rng = np.random.default_rng(11)
    k = np.stack([rays["kx"], rays["ky"], rays["kz"]], 1)
    b = rng.normal(size=(n, 3))
    p = b - np.sum(b * k, 1)[:, None] * k
    rp = dict(rays, px=p[:, 0], py=p[:, 1], pz=p[:, 2])
    _, _, tu, _ = ob.trace_rays(s, rays, seed=21)
    _, _, tp, _ = ob.trace_rays(s, rp, seed=22)
    for key in ("det_hits", "absorbed"):
        x, y = tu[key], tp[key]
        z = (x - y) / math.sqrt(x + y)
        assert abs(z) < 4.5, (key, x, y)
    h1, h2 = np.array(tu["refl_hist"][:4]), np.array(tp["refl_hist"][:4])
    z = (h1 - h2) / np.sqrt(h1 + h2 + 1)
    assert np.all(np.abs(z) < 4.5), (h1, h2)


def _rays_of_source(src, n, seed):
    """rays that a zero-cone, zero-spot mono source along src's axis emits"""
    ax = np.asarray(src["axis"], float)
    ax = ax / np.linalg.norm(ax)
    o = np.asarray(src["origin_mm"], float)
    rng = np.random.default_rng(seed)
    # small direction spread so that the rays sample the rocking curve
    d = ax[None, :] + rng.normal(scale=2e-3, size=(n, 3))
    return dict(ox=np.full(n, o[0]), oy=np.full(n, o[1]), oz=np.full(n, o[2]),
                kx=d[:, 0], ky=d[:, 1], kz=d[:, 2], E=np.full(n, src["components"][0]["e0_keV"]))


@pytest.mark.parametrize("pol", [None, [0.0, 1.0, 0.3]])
def test_user_rays_equal_a_zero_cone_source(pol):
    w = W.flat_hopg_mono()
    s = w["spec"]
    src = dict(w["source"], cone_half_angle_rad=0.0, spot_fwhm_mm=(0.0, 0.0))
    if pol is not None:
        src["polarization"] = pol
    n = 20_000
    img, tal, rec = ob.trace(s, src, n, seed=5, ray_offset=100, records=True)
    ax = np.asarray(src["axis"], float)
    ax /= np.linalg.norm(ax)
    o = src["origin_mm"]
    rays = dict(ox=np.full(n, o[0]), oy=np.full(n, o[1]), oz=np.full(n, o[2]),
                kx=np.full(n, ax[0]), ky=np.full(n, ax[1]), kz=np.full(n, ax[2]),
                E=np.full(n, src["components"][0]["e0_keV"]))
    if pol is not None:
        rays.update(px=np.full(n, pol[0]), py=np.full(n, pol[1]), pz=np.full(n, pol[2]))
    img2, _, tal2, rec2 = ob.trace_rays(s, rays, seed=5, ray_offset=100, records=True)
    assert np.array_equal(img, img2)
    assert tal == tal2
    for f in ("ray_id", "outcome", "nrefl", "ncoll", "ix", "iy"):
        assert np.array_equal(rec[f], rec2[f]), f
    assert np.allclose(rec["pos"], rec2["pos"], rtol=0, atol=1e-9)
    assert np.allclose(rec["pol"], rec2["pol"], rtol=0, atol=1e-12)
    if pol is not None:
        assert np.all(np.abs(np.linalg.norm(rec["pol"], axis=1) - 1) < 1e-12)
        assert np.all(np.abs(np.sum(rec["pol"] * rec["dir"], 1)) < 1e-12)
    else:
        assert not rec["pol"].any()


def test_user_rays_degenerate_inputs():
    s = W.flat_hopg_mono()["spec"]
    src = W.flat_hopg_mono()["source"]
    o, ax = src["origin_mm"], src["axis"]
    rays = dict(ox=np.array([o[0]] * 4), oy=np.array([o[1]] * 4), oz=np.array([o[2]] * 4),
                kx=np.array([0.0, ax[0], ax[0], ax[0]]), ky=np.array([0.0, ax[1], ax[1], ax[1]]),
                kz=np.array([0.0, ax[2], ax[2], ax[2]]), E=np.array([8.0, -1.0, np.nan, 8.0]))
    _, _, t, rec = ob.trace_rays(s, rays, seed=1, records=True)
    # zero direction, negative and NaN energies cannot enter; the last ray does
    assert list(rec["outcome"][:3]) == [0, 0, 0]
    assert rec["outcome"][3] != 0
    assert t["emitted"] == 4 and t["miss"] == 3
    _, _, t0, _ = ob.trace_rays(s, {k: v[:0] for k, v in rays.items()}, seed=1)
    assert t0["emitted"] == 0 and t0["det_hits"] == 0
    with pytest.raises(RuntimeError):
        ob.trace_rays(s, dict(rays, px=rays["kx"]), seed=1)        # partial polarisation arrays
