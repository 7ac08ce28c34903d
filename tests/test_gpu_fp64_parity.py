"""FP64 CUDA path vs the FP64 CPU oracle, ray by ray on the same Philox
streams, through the C ABI.  Tolerance: outcomes, reflection and collision
counts identical; positions, directions and detector coordinates within 1e-9
relative (scale max(|x|, 1 mm)); integer images identical except rays whose
oracle pixel coordinate is within 1e-9 of a pixel edge."""
import math

import numpy as np
import pytest

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-9


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16955_gb300 as H
    return H


def _near_edge(rec, spec):
    fx = rec["u_mm"] / spec["pixel_mm"] + 0.5 * spec["det_nx"]
    fy = rec["v_mm"] / spec["pixel_mm"] + 0.5 * spec["det_ny"]
    ex = np.abs(fx - np.round(fx)) <= REL * np.maximum(np.abs(fx), 1.0)
    ey = np.abs(fy - np.round(fy)) <= REL * np.maximum(np.abs(fy), 1.0)
    return ex | ey


def compare(H, spec, source, n, seed, offset=0):
    import torch
    s = H.heart_spectrometer_create(spec)
    dt = torch.int64 if spec.get("count_type") == "i64" else torch.int32
    img = torch.zeros(s.shape, dtype=dt, device="cuda")
    g, gt = H.heart_trace_records(s, source, n, seed, offset, precision="fp64", d_image=img)
    o_img, ot, o = ob.trace(spec, source, n, seed, ray_offset=offset, records=True)
    s.close()
    assert np.array_equal(g["ray_id"], o["ray_id"])
    bad = np.flatnonzero((g["outcome"] != o["outcome"]) | (g["nrefl"] != o["nrefl"]) |
                         (g["ncoll"] != o["ncoll"]))
    assert bad.size == 0, ("decision mismatch", bad[:5], g[bad[:2]], o[bad[:2]])
    for f in ("pos", "dir"):
        scale = np.maximum(np.abs(o[f]), 1.0)
        assert np.all(np.abs(g[f] - o[f]) <= REL * scale), f
    assert np.allclose(g["energy_keV"], o["energy_keV"], rtol=1e-13, atol=0)
    hit = ~np.isnan(o["u_mm"])
    assert np.array_equal(hit, ~np.isnan(g["u_mm"]))
    for f in ("u_mm", "v_mm"):
        scale = np.maximum(np.abs(o[f][hit]), 1.0)
        assert np.all(np.abs(g[f][hit] - o[f][hit]) <= REL * scale), f
    pix_bad = (g["ix"] != o["ix"]) | (g["iy"] != o["iy"])
    edge = _near_edge(o, spec)
    assert np.all(edge[pix_bad]), "pixel mismatch away from a pixel edge"
    assert pix_bad.sum() <= max(1, int(1e-6 * n))
    gi = img.cpu().numpy().astype(np.int64)
    assert int(np.abs(gi - o_img).sum()) <= 2 * int(pix_bad.sum())
    for k in ("emitted", "miss", "absorbed", "exit_front", "exit_back", "exit_side", "capped", "stuck",
              "no_bragg", "collisions", "refl_hist"):
        assert gt[k] == ot[k], k
    return g, gt


@pytest.mark.parametrize("sampler", ["thinned", "plain"])
def test_flat_hopg_mono_replays_oracle(H, sampler):
    w = W.flat_hopg_mono()
    g, t = compare(H, dict(w["spec"], sampler=sampler), w["source"], 40_000, w["seed"])
    assert t["det_hits"] > 50 and t["exit_front"] > 200


@pytest.mark.parametrize("sampler", ["thinned", "plain"])
def test_von_hamos_polychromatic_replays_oracle(H, sampler):
    w = W.von_hamos_hapg()
    g, t = compare(H, dict(w["spec"], sampler=sampler), w["source"], 40_000, w["seed"], offset=123_456_789_000)
    assert t["exit_front"] > 30


@pytest.mark.parametrize("mdf", ["lorentzian", "pseudo_voigt", "vmf", "wl", "swl", "uniform"])
def test_each_mosaic_distribution(H, mdf):
    w = W.flat_hopg_mono()
    s = dict(w["spec"])
    s.update(mdf=mdf, mdf_eta=0.3, mdf_fwhm_rad=0.2 * W.DEG)
    compare(H, s, w["source"], 15_000, 7)


@pytest.mark.parametrize("irc,extra", [("darwin_prins", {"prins_g": 0.05}),
                                       ("pseudo_voigt", {"irc_fwhm_rad": 50e-6, "irc_lorentz_fwhm_rad": 8e-6}),
                                       ("gaussian", {}), ("lorentzian", {}), ("box", {})])
def test_each_rocking_curve(H, irc, extra):
    w = W.von_hamos_hapg()
    s = dict(w["spec"])
    s.update(irc=irc, **extra)
    compare(H, s, w["source"], 15_000, 8)


def test_spectral_components_and_spot(H):
    w = W.flat_hopg_mono()
    src = dict(w["source"])
    src.update(components=[dict(kind="lorentz", e0_keV=8.0, width_keV=0.01, weight=1.0),
                           dict(kind="uniform", lo_keV=7.9, hi_keV=8.1, weight=0.5),
                           dict(kind="inv_e", lo_keV=7.5, hi_keV=8.5, weight=0.5),
                           dict(kind="gauss", e0_keV=8.05, width_keV=0.02, weight=1.0)],
               spot_fwhm_mm=(0.3, 0.7))
    compare(H, w["spec"], src, 15_000, 9)


def test_cap_stuck_and_no_bragg(H):
    w = W.flat_hopg_mono()
    s = dict(w["spec"])
    s.update(max_reflections=0, max_collisions=20)
    src = dict(w["source"])
    src.update(components=[dict(kind="mono", e0_keV=8.0, weight=1.0), dict(kind="mono", e0_keV=1.5, weight=0.2)])
    g, t = compare(H, s, src, 10_000, 10)
    assert t["capped"] > 0 and t["stuck"] > 0 and t["no_bragg"] > 0


def test_int64_image_and_empty_trace(H):
    import torch
    w = W.flat_hopg_mono()
    s = dict(w["spec"])
    s["count_type"] = "i64"
    compare(H, s, w["source"], 5_000, 11)
    sp = H.heart_spectrometer_create(s)
    img = torch.zeros(sp.shape, dtype=torch.int64, device="cuda")
    t = H.heart_trace(sp, w["source"], 0, 1, 0, img, precision="fp64")
    assert t["emitted"] == 0 and int(img.sum()) == 0
    sp.close()


def test_invalid_descriptors_rejected_before_launch(H):
    import torch
    w = W.flat_hopg_mono()
    for bad in ({"thickness_mm": -1.0}, {"mdf_fwhm_rad": 0.0}, {"det_nx": 0}, {"normal": [0.0, 0.0, 0.0]},
                {"axis": [0.0, 0.0, 1.0]}):
        s = dict(w["spec"])
        s.update(bad)
        with pytest.raises(H.HeartError) as e:
            H.heart_spectrometer_create(s)
        assert e.value.status == 1
    sp = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(sp.shape, dtype=torch.int32, device="cuda")
    src = dict(w["source"])
    src["components"] = []
    with pytest.raises(H.HeartError):
        H.heart_trace(sp, src, 10, 1, 0, img, precision="fp64")
    src = dict(w["source"])
    src["cone_half_angle_rad"] = -1.0
    with pytest.raises(H.HeartError):
        H.heart_trace(sp, src, 10, 1, 0, img, precision="fp64")
    # a misaligned image pointer is refused
    raw = torch.zeros(sp.shape[0] * sp.shape[1] + 1, dtype=torch.int32, device="cuda")
    view = raw.view(torch.uint8)[2:2 + 4 * sp.shape[0] * sp.shape[1]]
    with pytest.raises(H.HeartError):
        H.heart_trace(sp, w["source"], 10, 1, 0, view, precision="fp64")
    sp.close()


def test_host_buffer_path_equals_device_path(H):
    import torch
    w = W.flat_hopg_mono()
    sp = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(sp.shape, dtype=torch.int32, device="cuda")
    t1 = H.heart_trace(sp, w["source"], 20_000, 3, 0, img, precision="fp64")
    h = np.ones(sp.shape, dtype=np.int32)
    t2 = H.heart_trace_host(sp, w["source"], 20_000, 3, 0, h, precision="fp64")
    assert t1 == t2
    assert np.array_equal(h - 1, img.cpu().numpy())
    sp.close()
