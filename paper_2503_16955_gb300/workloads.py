"""Seeded synthetic spectrometer workloads (inputs only).

This module builds the neutral parameter dictionaries that both the GPU
library binding and the CPU oracle binding accept.  It contains no part of the
ray-transport arithmetic: the only physics used is Bragg's law to *place*
crystal, source and detector (a spectrometer is aligned for its central
energy), exactly as an experimenter would.

Units: mm, keV, rad.  Graphite (002): d = 3.354 Angstrom.

Workloads (the paper's set-ups, Sec. 4, with synthetic spectra because the
measured ones are not available):
  flat_hopg_mono        flat HOPG, 100 um, Gaussian mosaic 0.4 deg, Darwin IRC
                        20 urad, mono 8 keV point source 300 mm away, 2 deg cone,
                        256^2 x 50 um detector at the specular image point,
                        max 3 reflections, 2e5 rays, int32.
  von_hamos_hapg        cylindrical HAPG R = 80 mm, 40 um, pseudo-Voigt mosaic
                        0.1 deg (eta 0.5), Darwin-Prins IRC 20 urad (g = 0.05),
                        three Gaussian lines 7.8/8.0/8.2 keV on a 1/E continuum,
                        0.5 mm spot, 1024^2 x 50 um detector, max 5 reflections.
  batched_64            64 spectrometers drawn from seed 3.
  serving_stream        Poisson stream of trace jobs drawn like batched_64.
  von_hamos_large       cylindrical HAPG R = 100 mm, 100 um, Lorentzian mosaic
                        0.2 deg, pseudo-Voigt IRC 50/8 urad, elastic 8.5 keV +
                        inelastic 8.45 keV lines, 4096^2 x 25 um, int64.
"""
import math

import numpy as np

HC_KEV_A = 12.398419843320026
D_GRAPHITE_A = 3.354
DEG = math.pi / 180.0


def bragg_angle(E_keV, d_A=D_GRAPHITE_A):
    """Alignment helper: the Bragg angle used to position components."""
    return math.asin(HC_KEV_A / (2.0 * d_A * E_keV))


def _unit(v):
    v = np.asarray(v, dtype=float)
    return (v / np.linalg.norm(v)).tolist()


def _base_crystal():
    return dict(
        d_spacing_A=D_GRAPHITE_A,
        absorption_ref_keV=8.0,
        absorption_power=0.0,
        refl_K_per_mm2=-1.0,            # derive from the Darwin width below
        refl_darwin_fwhm_rad=20e-6,
        refl_ref_keV=8.0,
        irc_shift_rad=0.0,
        prins_g=0.0,
        irc_lorentz_fwhm_rad=0.0,
        mdf_eta=0.0,
        max_collisions=1_000_000,
        count_type="i32",
    )


def flat_layout(E0, dist_mm=300.0, det_dist_mm=300.0, size=(120.0, 40.0), thickness=0.1):
    """Flat crystal in the z = 0 plane (normal +z, dispersion along x), source at
    grazing angle aB(E0) at dist_mm from the crystal centre, detector centred on
    the central reflected ray det_dist_mm past the crystal, facing it."""
    aB = bragg_angle(E0)
    ca, sa = math.cos(aB), math.sin(aB)
    spec = _base_crystal()
    spec.update(geometry="flat", thickness_mm=thickness, radius_mm=0.0,
                centre_mm=[0.0, 0.0, 0.0], normal=[0.0, 0.0, 1.0], axis=[1.0, 0.0, 0.0],
                centre_axial_mm=0.0, size_disp_mm=size[0], size_nondisp_mm=size[1],
                det_centre_mm=[det_dist_mm * ca, 0.0, det_dist_mm * sa],
                det_u=[sa, 0.0, -ca], det_v=[0.0, 1.0, 0.0])
    origin = [-dist_mm * ca, 0.0, dist_mm * sa]
    axis = [ca, 0.0, -sa]
    return spec, origin, axis


def cyl_layout(E0, R, size=(80.0, 30.0), thickness=0.04, det_E0=None):
    """von Hamos: cylinder axis along x through the origin, source at the
    origin, crystal (inner face r = R) below the axis (centre direction -z),
    centred axially at R cot aB(E0); detector plane contains the axis, centred
    at the axial focus 2 R cot aB(det_E0), u along the axis."""
    aB = bragg_angle(E0)
    zc = R / math.tan(aB)
    aD = bragg_angle(det_E0 if det_E0 is not None else E0)
    spec = _base_crystal()
    spec.update(geometry="cyl", thickness_mm=thickness, radius_mm=R,
                centre_mm=[0.0, 0.0, 0.0], normal=[0.0, 0.0, -1.0], axis=[1.0, 0.0, 0.0],
                centre_axial_mm=zc, size_disp_mm=size[0], size_nondisp_mm=size[1],
                det_centre_mm=[2.0 * R / math.tan(aD), 0.0, 0.0],
                det_u=[1.0, 0.0, 0.0], det_v=[0.0, 1.0, 0.0])
    origin = [0.0, 0.0, 0.0]
    centre_pt = np.array([zc, 0.0, -R])
    axis = _unit(centre_pt)
    # cone half-angle: the crystal's angular radius seen from the source + 10 %
    half = 0.5 * size[1] / R
    worst = 0.0
    for z in (zc - 0.5 * size[0], zc + 0.5 * size[0]):
        for ph in (-half, half):
            p = np.array([z, R * math.sin(ph), -R * math.cos(ph)])
            c = float(np.dot(p / np.linalg.norm(p), axis))
            worst = max(worst, math.acos(min(1.0, c)))
    return spec, origin, axis, 1.1 * worst


def flat_hopg_mono(n_rays=200_000, seed=1):
    """Plain FP64 single-configuration case (flat HOPG, mono 8 keV)."""
    E0 = 8.0
    spec, origin, axis = flat_layout(E0, size=(120.0, 40.0), thickness=0.1)
    spec.update(mdf="gaussian", mdf_fwhm_rad=0.4 * DEG, irc="darwin", irc_fwhm_rad=20e-6,
                absorption_length_mm=2.0, max_reflections=3,
                det_nx=256, det_ny=256, pixel_mm=0.05, count_type="i32")
    src = dict(components=[dict(kind="mono", e0_keV=E0, weight=1.0)], origin_mm=origin,
               axis=axis, cone_half_angle_rad=2.0 * DEG, spot_fwhm_mm=(0.0, 0.0))
    return dict(name="flat_hopg_mono", spec=spec, source=src, n_rays=n_rays, seed=seed)


def _three_line_spectrum(scale=1.0):
    lines = [(7.8, 0.2), (8.0, 0.5), (8.2, 0.3)]
    comps = [dict(kind="gauss", e0_keV=e * scale, width_keV=0.005 * scale, weight=0.9 * w)
             for e, w in lines]
    comps.append(dict(kind="inv_e", lo_keV=7.5 * scale, hi_keV=8.5 * scale, weight=0.1))
    return comps


def von_hamos_hapg(n_rays=100_000_000, seed=2):
    """Cylindrical HAPG, polychromatic source (FP32 bulk vs FP64)."""
    E0 = 8.0
    spec, origin, axis, cone = cyl_layout(E0, 80.0, size=(80.0, 30.0), thickness=0.04)
    spec.update(mdf="pseudo_voigt", mdf_fwhm_rad=0.1 * DEG, mdf_eta=0.5,
                irc="darwin_prins", irc_fwhm_rad=20e-6, prins_g=0.05,
                absorption_length_mm=2.0, absorption_ref_keV=8.0, absorption_power=3.0,
                max_reflections=5, det_nx=1024, det_ny=1024, pixel_mm=0.05, count_type="i32")
    src = dict(components=_three_line_spectrum(), origin_mm=origin, axis=axis,
               cone_half_angle_rad=cone, spot_fwhm_mm=(0.5, 0.5))
    return dict(name="von_hamos_hapg", spec=spec, source=src, n_rays=n_rays, seed=seed)


def von_hamos_large(n_rays=10_000_000_000, seed=5):
    """Large streamed job: R = 100 mm HAPG, elastic + inelastic lines, int64."""
    spec, origin, axis, cone = cyl_layout(8.45, 100.0, size=(80.0, 30.0), thickness=0.1,
                                          det_E0=8.45)
    spec.update(mdf="lorentzian", mdf_fwhm_rad=0.2 * DEG, irc="pseudo_voigt",
                irc_fwhm_rad=50e-6, irc_lorentz_fwhm_rad=8e-6,
                absorption_length_mm=2.0, absorption_ref_keV=8.0, absorption_power=3.0,
                max_reflections=8, det_nx=4096, det_ny=4096, pixel_mm=0.025, count_type="i64")
    comps = [dict(kind="gauss", e0_keV=8.5, width_keV=0.003, weight=0.25),
             dict(kind="gauss", e0_keV=8.45, width_keV=0.030, weight=0.75)]
    src = dict(components=comps, origin_mm=origin, axis=axis, cone_half_angle_rad=cone,
               spot_fwhm_mm=(0.0, 0.0))
    return dict(name="von_hamos_large", spec=spec, source=src, n_rays=n_rays, seed=seed)


def random_spectrometer(rng, ray_range=(1e5, 1e8)):
    """One spectrometer of the batched / serving mix."""
    hapg = rng.random() < 0.5
    cyl = rng.random() < 0.5
    R = float(rng.uniform(50.0, 200.0))
    t = float(math.exp(rng.uniform(math.log(0.020), math.log(0.200))))
    mdf = ["gaussian", "lorentzian", "pseudo_voigt"][int(rng.integers(0, 3))]
    eta = float(rng.uniform(0.0, 1.0))
    fw = float(math.exp(rng.uniform(math.log(0.05), math.log(0.5)))) * DEG
    Ec = float(rng.uniform(5.0, 12.0))
    n = int(round(math.exp(rng.uniform(math.log(ray_range[0]), math.log(ray_range[1])))))
    side = [512, 1024, 2048][int(rng.integers(0, 3))]
    if cyl:
        spec, origin, axis, cone = cyl_layout(Ec, R, size=(80.0, 30.0), thickness=t)
    else:
        spec, origin, axis = flat_layout(Ec, size=(80.0, 30.0), thickness=t)
        # cone: the crystal's angular radius seen from 300 mm + 10 %
        corners = [np.array([x, y, 0.0]) for x in (-40.0, 40.0) for y in (-15.0, 15.0)]
        o = np.array(origin)
        worst = max(math.acos(min(1.0, float(np.dot((c - o) / np.linalg.norm(c - o), axis))))
                    for c in corners)
        cone = 1.1 * worst
    spec.update(mdf=mdf, mdf_fwhm_rad=fw, mdf_eta=eta if mdf == "pseudo_voigt" else 0.0,
                irc="pseudo_voigt", irc_fwhm_rad=50e-6, irc_lorentz_fwhm_rad=8e-6,
                absorption_length_mm=2.0, absorption_ref_keV=8.0, absorption_power=3.0,
                max_reflections=5, det_nx=side, det_ny=side, pixel_mm=0.05, count_type="i32",
                crystal_kind="HAPG" if hapg else "HOPG")
    src = dict(components=_three_line_spectrum(Ec / 8.0), origin_mm=origin, axis=axis,
               cone_half_angle_rad=cone, spot_fwhm_mm=(0.5, 0.5))
    return dict(spec=spec, source=src, n_rays=n, E_c=Ec)


def batched_64(seed=3, n_configs=64, ray_range=(1e5, 1e8)):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n_configs):
        j = random_spectrometer(rng, ray_range)
        j["seed"] = 1000 + i
        jobs.append(j)
    return jobs


def serving_stream(seed=4, n_jobs=10_000, rate_per_s=200.0, ray_range=(1e4, 1e8)):
    """Poisson arrivals; each job drawn like the batched mix."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        j = random_spectrometer(rng, ray_range)
        j["seed"] = 50_000 + i
        j["arrival_s"] = t
        jobs.append(j)
    return jobs


def user_rays(workload, n, seed, polarised=False, e_sigma_keV=0.15):
    """Seeded user-supplied rays for a workload (Sec. 2.1's ray arrays): origins
    in the source spot, directions uniform over a disc of the cone's half angle
    around its axis, energies Gaussian about the first line, optional random
    linear polarisations (not yet perpendicular to the rays).  Also a few
    degenerate rays: index 0 has a zero direction, index 1 a negative energy.
    Returns a dict of float64 arrays ox, oy, oz, kx, ky, kz, E (px, py, pz)."""
    src = workload["source"]
    rng = np.random.default_rng(seed)
    ax = np.array(_unit(src["axis"]))
    t = np.array([1.0, 0.0, 0.0]) if abs(ax[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    b1 = np.array(_unit(np.cross(ax, t)))
    b2 = np.cross(ax, b1)
    cone = max(src["cone_half_angle_rad"], 1e-3)
    r = cone * np.sqrt(rng.uniform(size=n))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    d = ax[None, :] + (r * np.cos(phi))[:, None] * b1 + (r * np.sin(phi))[:, None] * b2
    sig = np.asarray(src.get("spot_fwhm_mm", (0.0, 0.0)), float) / 2.3548200450309493
    o = np.asarray(src["origin_mm"], float)[None, :] + \
        (sig[0] * rng.normal(size=n))[:, None] * b1 + (sig[1] * rng.normal(size=n))[:, None] * b2
    e0 = src["components"][0].get("e0_keV") or 0.5 * (src["components"][0]["lo_keV"] +
                                                      src["components"][0]["hi_keV"])
    E = e0 + e_sigma_keV * rng.normal(size=n)
    if n > 0:
        d[0] = 0.0
    if n > 1:
        E[1] = -1.0
    out = dict(ox=o[:, 0].copy(), oy=o[:, 1].copy(), oz=o[:, 2].copy(),
               kx=d[:, 0].copy(), ky=d[:, 1].copy(), kz=d[:, 2].copy(), E=E)
    if polarised:
        p = rng.normal(size=(n, 3))
        out.update(px=p[:, 0].copy(), py=p[:, 1].copy(), pz=p[:, 2].copy())
    return out


def scaled(workload, n_rays):
    """Same workload with a different ray count."""
    w = dict(workload)
    w["n_rays"] = int(n_rays)
    return w
