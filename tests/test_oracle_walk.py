"""Pins of the oracle's ray path: hand-traced walks with injected random words,
closed-form transport laws, quadrature of the paper's cross-section, the
Appendix's psi distribution, focusing geometry, invariants."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

LN2 = math.log(2.0)


def flat(**kw):
    # the plain walk: the hand-traced rays below inject its word layout
    s = dict(W.flat_hopg_mono()["spec"], sampler="plain")
    s.update(kw)
    return s


def pencil(spec, alpha, E=8.0, dist=300.0):
    """mono point source aimed at the crystal centre at grazing angle alpha"""
    ca, sa = math.cos(alpha), math.sin(alpha)
    return dict(components=[dict(kind="mono", e0_keV=E, weight=1.0)],
                origin_mm=[-dist * ca, 0.0, dist * sa], axis=[ca, 0.0, -sa],
                cone_half_angle_rad=0.0, spot_fwhm_mm=(0.0, 0.0))


# --------------------------------------------------------------------------
# hand-traced single rays with injected words (4 words per free-path draw)
# --------------------------------------------------------------------------
TINY_STEP = 0xFFFFFFFF     # u0 = 1 - 2^-33: free path ~ 1e-10 / mubar
LONG_STEP = 0x00000000     # u0 = 2^-33: free path 22.87 / mubar
REJECT = 0xFFFFFFFF        # u1 ~ 1: not absorbed, v ~ 1 > any acceptance
ABSORB = 0x00000000        # u1 ~ 0 < mu0/mubar


def accept_word(spec, E):
    pa = ob.ray_constants(spec, E)["p_abs"]
    return int(math.ceil(pa * 2**32)) + 64        # just above the absorption share


def test_injected_exit_through_back_face():
    s = flat(thickness_mm=0.01)
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    k = [math.cos(aB), 0.0, -math.sin(aB)]
    rec = ob.walk_injected(s, 8.0, [1.0, 2.0, 0.0], k, [LONG_STEP, REJECT, 0, 0])
    assert ob.OUTCOME[int(rec["outcome"])] == "exit_back"
    L = 0.01 / math.sin(aB)
    assert np.allclose(rec["pos"], [1.0 + L * k[0], 2.0, -0.01], rtol=0, atol=1e-14)
    assert rec["ncoll"] == 0 and rec["nrefl"] == 0


def test_injected_absorption_at_free_path():
    s = flat()
    c = ob.ray_constants(s, 8.0)
    aB = c["alpha_B"]
    k = np.array([math.cos(aB), 0.0, -math.sin(aB)])
    w0 = 0x80000000
    rec = ob.walk_injected(s, 8.0, [0.0, 0.0, 0.0], k, [w0, ABSORB, 0, 0])
    assert ob.OUTCOME[int(rec["outcome"])] == "absorbed"
    l = -math.log((w0 + 0.5) / 2**32) / c["mubar"]
    assert np.allclose(rec["pos"], l * k, rtol=0, atol=1e-15)
    assert rec["ncoll"] == 1


def _mirror_case(s, words_after):
    c = ob.ray_constants(s, 8.0)
    aB = c["alpha_B"]
    k = np.array([math.cos(aB), 0.0, -math.sin(aB)])
    acc = accept_word(s, 8.0)
    # w2 = 0: crystallite normal within 5e-8 rad of the surface normal
    words = [TINY_STEP, acc, 0, 0] + words_after
    return k, ob.walk_injected(s, 8.0, [0.0, 0.0, 0.0], k.tolist(), words)


def test_injected_specular_reflection_then_front_exit_and_detector():
    s = flat()
    k, rec = _mirror_case(s, [LONG_STEP, REJECT, 0, 0])
    assert ob.OUTCOME[int(rec["outcome"])] == "exit_front"
    assert rec["nrefl"] == 1
    assert np.allclose(rec["dir"], [k[0], 0.0, -k[2]], atol=1e-6)
    # the detector hit, recomputed as a plain line-plane intersection
    x, d = np.array(rec["pos"]), np.array(rec["dir"])
    D0, eu, ev = (np.array(s[n]) for n in ("det_centre_mm", "det_u", "det_v"))
    nd = np.cross(eu, ev)
    t = np.dot(D0 - x, nd) / np.dot(d, nd)
    P = x + t * d - D0
    assert rec["u_mm"] == pytest.approx(np.dot(P, eu), abs=1e-9)
    assert rec["v_mm"] == pytest.approx(np.dot(P, ev), abs=1e-9)
    assert rec["ix"] == math.floor(rec["u_mm"] / 0.05 + 128)
    assert rec["iy"] == math.floor(rec["v_mm"] / 0.05 + 128)
    assert rec["det_hit"] == 1


def test_injected_double_reflection_restores_direction():
    s = flat()
    acc = accept_word(s, 8.0)
    k, rec = _mirror_case(s, [TINY_STEP, acc, 0, 0, LONG_STEP, REJECT, 0, 0])
    # second reflection off the same (H-bar side of the) planes: back downwards
    assert rec["nrefl"] == 2
    assert np.allclose(rec["dir"], k, atol=1e-6)


def test_injected_cap_and_stuck():
    s = flat(max_reflections=0)
    _, rec = _mirror_case(s, [LONG_STEP, REJECT, 0, 0])
    assert ob.OUTCOME[int(rec["outcome"])] == "capped" and rec["nrefl"] == 1
    s = flat(max_collisions=3)
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    k = [math.cos(aB), 0.0, -math.sin(aB)]
    rec = ob.walk_injected(s, 8.0, [0.0, 0.0, 0.0], k, [TINY_STEP, REJECT, 7, 9] * 10)
    assert ob.OUTCOME[int(rec["outcome"])] == "stuck" and rec["ncoll"] == 3


def test_injected_rocking_curve_rejects_off_bragg():
    # 200 urad away from the Bragg angle, the Darwin curve is ~1e-3 of its peak:
    # a candidate with v = 0.01 must be rejected, one with v ~ 1e-6 accepted
    s = flat(mdf="uniform", mdf_fwhm_rad=1e-9)
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + 200e-6
    k = [math.cos(a), 0.0, -math.sin(a)]
    pa = c["p_abs"]
    v_word = lambda v: int((pa + v * (1 - pa)) * 2**32)
    rec = ob.walk_injected(s, 8.0, [0, 0, 0], k, [TINY_STEP, v_word(0.01), 0, 0, LONG_STEP, REJECT, 0, 0])
    assert rec["nrefl"] == 0
    y = 200e-6 / (20e-6 * math.sqrt(2) / 3)
    Rrel = 1.0 / (y + math.sqrt(y * y - 1)) ** 2         # Darwin tail relative to the plateau
    c2 = math.cos(2 * a)
    P = Rrel * 0.5 * (1 + c2 * c2)
    rec = ob.walk_injected(s, 8.0, [0, 0, 0], k, [TINY_STEP, v_word(0.98 * P), 0, 0, LONG_STEP, REJECT, 0, 0])
    assert rec["nrefl"] == 1
    rec = ob.walk_injected(s, 8.0, [0, 0, 0], k, [TINY_STEP, v_word(1.02 * P), 0, 0, LONG_STEP, REJECT, 0, 0])
    assert rec["nrefl"] == 0


# --------------------------------------------------------------------------
# transport laws on a flat slab, pencil beam
# --------------------------------------------------------------------------
def test_beer_lambert_absorption_and_depth():
    s = flat(refl_K_per_mm2=0.0)             # no reflection: pure absorption
    a = 0.3
    n = 200_000
    img, tal, rec = ob.trace(s, pencil(s, a), n, seed=11, records=True)
    L = 0.1 / math.sin(a)
    p = 1 - math.exp(-0.5 * L)
    z = (tal["absorbed"] - n * p) / math.sqrt(n * p * (1 - p))
    assert abs(z) < 4.5
    assert tal["absorbed"] + tal["exit_back"] == n
    depth = -rec["pos"][rec["outcome"] == 1][:, 2]
    mu_z = 0.5 / math.sin(a)
    cdf = lambda d: (1 - np.exp(-mu_z * d)) / (1 - math.exp(-mu_z * 0.1))
    assert stats.kstest(depth, cdf).pvalue > 1e-3


@pytest.mark.parametrize("mdf,offset_G,extra", [
    ("gaussian", 0.2, {}),
    ("wl", 2.0, {"mdf_fwhm_rad": 0.063 * W.DEG}),
    ("lorentzian", 0.0, {"mdf_fwhm_rad": 0.1 * W.DEG}),
])
def test_first_reflection_probability_matches_cross_section_quadrature(mdf, offset_G, extra):
    s = flat(mdf=mdf, **extra)
    c = ob.ray_constants(s, 8.0)
    a = c["alpha_B"] + offset_G * s["mdf_fwhm_rad"]
    r = ob.reflection_rate(s, 8.0, a)             # quadrature of Eq. (ReflXsection)
    mu0 = c["mu0"]
    L = 0.1 / math.sin(a)
    p = r / (mu0 + r) * (1 - math.exp(-(mu0 + r) * L))
    n = 300_000
    _, tal, _ = ob.trace(s, pencil(s, a), n, seed=12)
    k = n - tal["refl_hist"][0]
    z = (k - n * p) / math.sqrt(n * p * (1 - p))
    assert abs(z) < 4.5, (k, n * p)


def test_vmf_rate_reduces_to_simple_zachariasen_form():
    # Sec. 2.2.3: for small Gamma the psi-integrated vMF gives Q G W(alpha - aB)
    G = 1e-3
    s = flat(mdf="vmf", mdf_fwhm_rad=G, irc="gaussian", irc_fwhm_rad=2e-7)
    c = ob.ray_constants(s, 8.0)
    aB = c["alpha_B"]
    for off in (0.0, 0.5 * G, 1.0 * G):
        r = ob.reflection_rate(s, 8.0, aB + off)
        c2 = math.cos(2 * aB)
        Gu = 0.5 * (1 + c2 * c2)
        W1 = math.sqrt(4 * LN2 / (math.pi * G * G)) * math.exp(-4 * LN2 * off * off / (G * G))
        assert r == pytest.approx(c["Q"] * Gu * W1, rel=3e-3)


# --------------------------------------------------------------------------
# crystallite orientation of accepted reflections (Appendix A)
# --------------------------------------------------------------------------
def test_accepted_psi_follows_method_II_not_method_I():
    G = 0.06 * W.DEG
    s = flat(mdf="lorentzian", mdf_fwhm_rad=G, irc="gaussian", irc_fwhm_rad=20e-6)
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    off = 3.0 * G
    a = aB + off
    _, psi = ob.sample_crystallites(s, 8.0, a, 15000, seed=5)
    edges = np.linspace(-12 * G, 12 * G, 25)
    inside = psi[(psi > edges[0]) & (psi < edges[-1])]
    hist = np.histogram(inside, edges)[0]

    def q_of_psi(p):
        return 2 * math.sin(off / 2) ** 2 + 2 * math.cos(a) * math.cos(aB) * math.sin(p / 2) ** 2

    def w_method2(p):                            # W(theta(psi)) dpsi
        return ob.mdf_W(s, q_of_psi(p))[0]

    def w_method1(p):                            # Eq. (Psi_From_Theta) extra factor
        S, Cc = math.sin(a) * math.sin(aB), math.cos(a) * math.cos(aB)
        j = math.sqrt(Cc * Cc * math.sin(p) ** 2 / (1 - (S + Cc * math.cos(p)) ** 2))
        return j * w_method2(p)

    def chi2_p(fn):
        mass = np.array([integrate.quad(fn, lo, hi, epsrel=1e-10)[0] for lo, hi in zip(edges[:-1], edges[1:])])
        exp = mass / mass.sum() * hist.sum()
        chi2 = ((hist - exp) ** 2 / exp).sum()
        return stats.chi2.sf(chi2, len(hist) - 1)

    assert chi2_p(w_method2) > 1e-3
    assert chi2_p(w_method1) < 1e-12


def test_accepted_delta_follows_rocking_curve():
    s = flat(mdf="gaussian", mdf_fwhm_rad=0.4 * W.DEG, irc="darwin", irc_fwhm_rad=20e-6)
    aB = ob.ray_constants(s, 8.0)["alpha_B"]
    d, _ = ob.sample_crystallites(s, 8.0, aB, 20000, seed=9)
    edges = np.linspace(-40e-6, 40e-6, 33)
    inside = d[(d > edges[0]) & (d < edges[-1])]
    hist = np.histogram(inside, edges)[0]
    mass = np.array([integrate.quad(lambda x: ob.irc(s, x)[0], lo, hi, epsrel=1e-10)[0]
                     for lo, hi in zip(edges[:-1], edges[1:])])
    exp = mass / mass.sum() * hist.sum()
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2, len(hist) - 1) > 1e-3


# --------------------------------------------------------------------------
# focusing geometry
# --------------------------------------------------------------------------
@pytest.mark.parametrize("E", [7.9, 8.0, 8.1])
def test_von_hamos_line_at_twice_R_cot_bragg(E):
    w = W.von_hamos_hapg()
    s = dict(w["spec"])
    s.update(thickness_mm=0.01, mdf="gaussian", mdf_fwhm_rad=0.1 * W.DEG, irc="darwin",
             det_nx=1024, det_ny=256, pixel_mm=0.05)
    src = dict(w["source"])
    src.update(components=[dict(kind="mono", e0_keV=E, weight=1.0)], spot_fwhm_mm=(0.0, 0.0))
    img, tal, _ = ob.trace(s, src, 1_000_000, seed=21)
    R = s["radius_mm"]
    want = 2 * R / math.tan(W.bragg_angle(E)) - s["det_centre_mm"][0]
    col = img.sum(axis=0)
    assert col.sum() > 300
    u_mode = (np.argmax(col) + 0.5 - 512) * 0.05
    assert abs(u_mode - want) <= 0.1, (u_mode, want)


def test_flat_crystal_mosaic_focus_at_detector_centre():
    w = W.flat_hopg_mono()
    s = dict(w["spec"])
    s.update(thickness_mm=0.01, mdf_fwhm_rad=0.1 * W.DEG)
    img, tal, _ = ob.trace(s, w["source"], 400_000, seed=23)
    col = img.sum(axis=0)
    assert col.sum() > 100
    assert abs(np.argmax(col) - 127.5) <= 1


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
def _conserved(t):
    return t["emitted"] == (t["miss"] + t["absorbed"] + t["exit_front"] + t["exit_back"] +
                            t["exit_side"] + t["capped"] + t["stuck"])


def test_conservation_and_thread_and_shard_invariance():
    w = W.von_hamos_hapg()
    n = 30_000
    img1, t1, _ = ob.trace(w["spec"], w["source"], n, seed=2, n_threads=1)
    img8, t8, _ = ob.trace(w["spec"], w["source"], n, seed=2, n_threads=8)
    assert _conserved(t1) and t1 == t8 and np.array_equal(img1, img8)
    a, ta, _ = ob.trace(w["spec"], w["source"], n // 3, seed=2, ray_offset=0)
    b, tb, _ = ob.trace(w["spec"], w["source"], n - n // 3, seed=2, ray_offset=n // 3)
    assert np.array_equal(a + b, img1)
    assert t1["det_hits"] == ta["det_hits"] + tb["det_hits"] == img1.sum()
    assert t1["det_hits"] <= t1["exit_front"] + t1["exit_back"] + t1["exit_side"]
    assert sum(t1["refl_hist"]) == n - t1["miss"]


def test_source_words_come_from_their_philox_blocks():
    # Sec. 2.1 draws energy, direction and spot as independent uniforms; which Philox
    # word feeds which draw is a convention: call 0 holds the spot's radius and angle
    # and the direction's 1 - cos(phi) and azimuth, call 1 the component, its parameter
    # and the Gaussian line's pair.  Checked on each ray against the published
    # generator's words (counter = (ray, 0, call, 0), key = seed), with the crystal
    # turned away so that every record keeps the sampled origin, direction and energy.
    s = flat(normal=[0.0, 0.0, -1.0])
    axis = np.array([0.3, -0.2, 0.9])
    axis /= np.linalg.norm(axis)
    origin = np.array([1.0, 2.0, 3.0])
    fwhm, half = 0.8, 0.05
    comps = [dict(kind="uniform", lo_keV=7.0, hi_keV=7.2, weight=0.3),
             dict(kind="uniform", lo_keV=9.0, hi_keV=9.4, weight=0.7)]
    src = dict(components=comps, origin_mm=origin.tolist(), axis=axis.tolist(),
               cone_half_angle_rad=half, spot_fwhm_mm=(fwhm, fwhm))
    n, seed = 3000, 0x1234_5678_9ABC
    _, tal, rec = ob.trace(s, src, n, seed=seed, records=True)
    assert tal["miss"] == n
    key = (seed & 0xFFFFFFFF, seed >> 32)
    sigma = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    one_minus_cos = 2.0 * math.sin(0.5 * half) ** 2

    def u(w):
        return (w + 0.5) / 2.0 ** 32

    for i in range(n):
        a = ob.philox((i, 0, 0, 0), key)
        b = ob.philox((i, 0, 1, 0), key)
        # energy: component by word 0 of call 1 against the cumulative weight, then
        # uniform on its range by word 1
        lo, hi = (7.0, 7.2) if u(b[0]) < 0.3 else (9.0, 9.4)
        assert rec["energy_keV"][i] == pytest.approx(lo + (hi - lo) * u(b[1]), rel=1e-13)
        # direction: 1 - cos(phi) is uniform on [0, 1 - cos(half-angle)] by word 2 of call 0
        k = rec["dir"][i]
        assert 1.0 - float(np.dot(k, axis)) == pytest.approx(u(a[2]) * one_minus_cos, rel=1e-9, abs=1e-14)
        # spot (circular): the offset's length is the Box-Muller radius of word 0 of call 0
        d = rec["pos"][i] - origin
        assert abs(float(np.dot(d, axis))) <= 1e-12
        assert float(np.dot(d, d)) / sigma ** 2 == pytest.approx(-2.0 * math.log(u(a[0])), rel=1e-9, abs=1e-12)
    # ray ids across 2^32: the counter's first two words are the id's low and high halves
    off = (1 << 32) - 100
    _, _, rec = ob.trace(s, src, 200, seed=seed, ray_offset=off, records=True)
    for i in range(200):
        ray = off + i
        assert int(rec["ray_id"][i]) == ray
        b = ob.philox((ray & 0xFFFFFFFF, ray >> 32, 1, 0), key)
        lo, hi = (7.0, 7.2) if u(b[0]) < 0.3 else (9.0, 9.4)
        assert rec["energy_keV"][i] == pytest.approx(lo + (hi - lo) * u(b[1]), rel=1e-13)


def test_source_sampling_distributions():
    # crystal turned away from the source: every ray misses and its record keeps
    # the sampled origin, direction and energy
    s = flat(normal=[0.0, 0.0, -1.0])
    comps = [dict(kind="gauss", e0_keV=8.0, width_keV=0.01, weight=0.5),
             dict(kind="inv_e", lo_keV=7.5, hi_keV=8.5, weight=0.3),
             dict(kind="uniform", lo_keV=7.0, hi_keV=7.2, weight=0.1),
             dict(kind="lorentz", e0_keV=9.0, width_keV=0.02, weight=0.1)]
    axis = np.array([0.3, -0.2, 0.9])
    axis /= np.linalg.norm(axis)
    src = dict(components=comps, origin_mm=[1.0, 2.0, 3.0], axis=axis.tolist(),
               cone_half_angle_rad=0.05, spot_fwhm_mm=(0.4, 1.0))
    n = 100_000
    _, tal, rec = ob.trace(s, src, n, seed=31, records=True)
    assert tal["miss"] == n
    E = rec["energy_keV"]

    def mix_cdf(x):
        x = np.asarray(x)
        return (0.5 * stats.norm.cdf(x, 8.0, 0.01)
                + 0.3 * np.clip(np.log(np.clip(x, 7.5, 8.5) / 7.5) / math.log(8.5 / 7.5), 0, 1)
                + 0.1 * np.clip((x - 7.0) / 0.2, 0, 1)
                + 0.1 * (stats.cauchy.cdf(x, 9.0, 0.01) - stats.cauchy.cdf(0, 9.0, 0.01))
                / (1 - stats.cauchy.cdf(0, 9.0, 0.01)))
    assert stats.kstest(E, mix_cdf).pvalue > 1e-3
    d = rec["dir"]
    cphi = d @ axis
    c0 = math.cos(0.05)
    assert stats.kstest(cphi, stats.uniform(loc=c0, scale=1 - c0).cdf).pvalue > 1e-3
    off = rec["pos"] - np.array([1.0, 2.0, 3.0])
    assert np.allclose(off @ axis, 0.0, atol=1e-12)
    spread = np.sort(np.linalg.svd(off, compute_uv=False) / math.sqrt(n))
    sig = np.array([0.4, 1.0]) / (2 * math.sqrt(2 * LN2))
    assert np.allclose(spread[1:], sig, rtol=0.01)


# --------------------------------------------------------------------------
# energy image and detector quantum efficiency (Sec. 2.3, Sec. 3)
# --------------------------------------------------------------------------
def test_qe_is_linear_interpolation_clamped_at_the_ends():
    table = [(7.5, 0.9), (8.0, 0.8), (8.6, 0.5), (9.0, 0.55)]
    xs, ys = zip(*table)
    for E in np.linspace(7.0, 9.5, 51):
        assert ob.qe_eval(table, E) == pytest.approx(np.interp(E, xs, ys), rel=1e-14, abs=1e-15)
    assert ob.qe_eval([], 8.0) == 1.0


def test_energy_image_sums_detected_photon_energies():
    w = W.von_hamos_hapg()
    qe = [(7.5, 0.9), (8.0, 0.8), (8.5, 0.5)]
    img, eimg, tal, rec = ob.trace_energy(w["spec"], w["source"], 40_000, 5, qe=qe, records=True)
    hit = rec["det_hit"] == 1
    assert int(img.sum()) == tal["det_hits"] == int(hit.sum())
    # per pixel: the sum of round(E * QE(E) * 1e6) over the rays binned there
    want = np.zeros_like(eimg)
    for r in rec[hit]:
        want[r["iy"], r["ix"]] += int(round(r["energy_keV"] * ob.qe_eval(qe, r["energy_keV"]) * 1e6))
    assert np.array_equal(eimg, want)
    # the count image is the plain trace's image, unchanged by the energy accumulator
    img2, _, _ = ob.trace(w["spec"], w["source"], 40_000, 5)
    assert np.array_equal(img, img2)


def test_mono_energy_image_is_count_times_energy():
    w = W.flat_hopg_mono()
    img, eimg, tal, _ = ob.trace_energy(w["spec"], w["source"], 100_000, 6)
    assert np.array_equal(eimg, img * 8_000_000)


# --------------------------------------------------------------------------
# tabulated spectrum (a density at knots; the CDF is linear between them)
# --------------------------------------------------------------------------
def _missing_source(comps, table=None):
    s = flat(normal=[0.0, 0.0, -1.0])          # every ray misses: records keep E
    src = dict(components=comps, origin_mm=[0.0, 0.0, 1.0], axis=[0.0, 0.0, 1.0],
               cone_half_angle_rad=0.01, spot_fwhm_mm=(0.0, 0.0))
    if table is not None:
        src["table"] = table
    return s, src


def test_tabulated_spectrum_follows_its_piecewise_linear_cdf():
    # an asymmetric table with a zero-density gap (7.9 - 8.0 keV) mixed with a line
    keV = np.array([7.6, 7.7, 7.9, 8.0, 8.05, 8.3])
    pdf = np.array([0.5, 2.0, 0.0, 0.0, 4.0, 1.0])
    s, src = _missing_source([dict(kind="table", weight=0.7), dict(kind="mono", e0_keV=9.0, weight=0.3)],
                             (keV, pdf))
    n = 200_000
    _, tal, rec = ob.trace(s, src, n, seed=41, records=True)
    E = rec["energy_keV"]
    tab = E[E < 8.5]
    assert abs(len(tab) / n - 0.7) < 5 * math.sqrt(0.21 / n)
    # CDF at the knots by hand (trapezoids), linear in between
    mass = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(keV))])
    cdf = lambda x: np.interp(x, keV, mass / mass[-1])
    assert stats.kstest(tab, cdf).pvalue > 1e-3
    assert not np.any((tab > 7.9) & (tab < 8.0))           # the empty interval is never drawn
    assert tab.min() >= 7.6 and tab.max() <= 8.3
    # the density within an interval is flat: fraction in [7.6, 7.65] vs [7.65, 7.7]
    a = np.count_nonzero((tab >= 7.6) & (tab < 7.65))
    b = np.count_nonzero((tab >= 7.65) & (tab < 7.7))
    assert abs(a - b) < 5 * math.sqrt(a + b)


def test_two_knot_table_reproduces_the_uniform_component():
    s, su = _missing_source([dict(kind="uniform", lo_keV=7.3, hi_keV=8.9, weight=1.0)])
    _, st = _missing_source([dict(kind="table", weight=1.0)], (np.array([7.3, 8.9]), np.array([2.5, 2.5])))
    _, _, ru = ob.trace(s, su, 20_000, seed=42, records=True)
    _, _, rt = ob.trace(s, st, 20_000, seed=42, records=True)
    assert np.array_equal(ru["energy_keV"], rt["energy_keV"])


def test_tabulated_spectrum_validation():
    s, src = _missing_source([dict(kind="table", weight=1.0)])
    for table in [None, (np.array([8.0]), np.array([1.0])), (np.array([8.0, 7.0]), np.array([1.0, 1.0])),
                  (np.array([7.0, 8.0]), np.array([1.0, -1.0])), (np.array([7.0, 8.0]), np.array([0.0, 0.0])),
                  (np.array([-1.0, 8.0]), np.array([1.0, 1.0]))]:
        bad = dict(src)
        if table is not None:
            bad["table"] = table
        with pytest.raises(RuntimeError):
            ob.trace(s, bad, 10, seed=1)
