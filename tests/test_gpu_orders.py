"""Higher-order reflections and the energy-dependent rocking curve through the
C ABI.  The FP64 kernel replays the oracle ray by ray (decisions identical,
positions within 1e-9 relative); the FP32 kernels follow the FP64 kernel on the
same streams within the usual budget (<= 1e-4 of rays flipped, hit positions
within 1 um) with an energy table, several orders (sampled and user rays,
polarised, no rocking curve), and one order given with its multiple; single,
batched, static and served FP32 traces of several orders agree exactly; rays
below the Bragg cutoff leave a cylinder where the FP64 kernel has them leave."""
import numpy as np
import pytest

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORDERS = [(1, 1.0, 1.0), (2, 0.45, 0.6), (3, 0.2, 0.4)]
TABLE = [(7.6, 0.8, -1e-5), (8.0, 1.0, 0.0), (8.4, 1.4, 2e-5)]


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16955_gb300 as H
    return H


def _replay(H, spec, src, n, seed):
    s = H.heart_spectrometer_create(spec)
    g, gt = H.heart_trace_records(s, src, n, seed, 0, precision="fp64")
    _, ot, o = ob.trace(spec, src, n, seed, records=True)
    s.close()
    bad = (g["outcome"] != o["outcome"]) | (g["nrefl"] != o["nrefl"]) | (g["ncoll"] != o["ncoll"])
    assert not bad.any(), np.flatnonzero(bad)[:5]
    scale = np.maximum(np.abs(o["pos"]), 1.0)
    assert np.all(np.abs(g["pos"] - o["pos"]) <= 1e-9 * scale)
    for k in ("emitted", "miss", "absorbed", "exit_front", "exit_back", "exit_side", "collisions", "refl_hist"):
        assert gt[k] == ot[k], k
    return gt


@pytest.mark.parametrize("sampler", ["thinned", "plain"])
def test_fp64_orders_and_energy_table_replay_oracle(H, sampler):
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], orders=ORDERS, irc_energy=TABLE, sampler=sampler)
    src = dict(w["source"], components=[dict(kind="uniform", lo_keV=7.5, hi_keV=16.5, weight=1.0)])
    t = _replay(H, spec, src, 60_000, 12)
    assert t["exit_front"] > 5


def test_fp64_second_order_equals_first_order_on_half_spacing(H):
    # order 2 on planes d is order 1 on planes d / 2 (Bragg's law on d / m) with
    # that order's K and width: at 16 keV the two spectrometers give the same
    # image on the same streams (plain sampler: the thinning bounds are not
    # computed the same way for the two descriptions)
    import torch
    w = W.von_hamos_hapg()
    base = dict(w["spec"], sampler="plain", refl_K_per_mm2=5.5e8)
    two = dict(base, orders=[(2, 4.0, 0.5)])       # order 2 alone: order 1 would change the majorant
    half = dict(base, d_spacing_A=base["d_spacing_A"] / 2, refl_K_per_mm2=2.2e9,
                irc_fwhm_rad=0.5 * base["irc_fwhm_rad"])
    src = dict(w["source"], components=[dict(kind="mono", e0_keV=16.0, weight=1.0)])
    imgs, tals = [], []
    for spec in (two, half):
        s = H.heart_spectrometer_create(spec)
        img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
        tals.append(H.heart_trace(s, src, 2_000_000, 4, 0, img, precision="fp64"))
        imgs.append(img.cpu().numpy())
        s.close()
    assert tals[0]["det_hits"] > 500
    diff = np.abs(imgs[0].astype(np.int64) - imgs[1]).sum()
    assert diff <= 2e-4 * tals[0]["det_hits"] + 2, diff
    assert abs(tals[0]["det_hits"] - tals[1]["det_hits"]) <= 1e-4 * tals[0]["det_hits"] + 1


def test_fp32_energy_table_follows_fp64(H):
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], irc_energy=TABLE)
    s = H.heart_spectrometer_create(spec)
    n = 200_000
    r64, t64 = H.heart_trace_records(s, w["source"], n, 6, 0, precision="fp64")
    r32, t32 = H.heart_trace_records(s, w["source"], n, 6, 0, precision="fp32")
    s.close()
    flip = (r64["outcome"] != r32["outcome"]) | (r64["nrefl"] != r32["nrefl"]) | (r64["ncoll"] != r32["ncoll"])
    assert flip.sum() <= max(2, 1e-4 * n), int(flip.sum())
    same = ~flip & (r64["det_hit"] == 1) & (r32["det_hit"] == 1)
    assert same.sum() > 100
    assert np.abs(r64["u_mm"][same] - r32["u_mm"][same]).max() <= 1e-3
    # the table changes the result: wider at high energy, shifted
    s0 = H.heart_spectrometer_create(w["spec"])
    r0, _ = H.heart_trace_records(s0, w["source"], n, 6, 0, precision="fp32")
    s0.close()
    assert np.count_nonzero(r0["nrefl"] != r32["nrefl"]) > 20


def _fp32_vs_fp64(H, spec, src, n, seed, min_hits=100):
    s = H.heart_spectrometer_create(spec)
    r64, t64 = H.heart_trace_records(s, src, n, seed, 0, precision="fp64")
    r32, t32 = H.heart_trace_records(s, src, n, seed, 0, precision="fp32")
    s.close()
    flip = (r64["outcome"] != r32["outcome"]) | (r64["nrefl"] != r32["nrefl"]) | (r64["ncoll"] != r32["ncoll"])
    assert flip.sum() <= max(2, 1e-4 * n), int(flip.sum())
    same = ~flip & (r64["det_hit"] == 1) & (r32["det_hit"] == 1)
    assert same.sum() >= min_hits, int(same.sum())
    assert np.abs(r64["u_mm"][same] - r32["u_mm"][same]).max() <= 1e-3
    assert np.abs(r64["v_mm"][same] - r32["v_mm"][same]).max() <= 1e-3
    assert t32["no_bragg"] == t64["no_bragg"]
    return r64, r32, t32


def _wide(w, lo=7.5, hi=16.5):
    return dict(w["source"], components=[dict(kind="uniform", lo_keV=lo, hi_keV=hi, weight=1.0)])


@pytest.mark.parametrize("sampler", ["thinned", "plain"])
def test_fp32_orders_follow_fp64_von_hamos(H, sampler):
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], orders=ORDERS, irc_energy=TABLE, sampler=sampler)
    r64, r32, t = _fp32_vs_fp64(H, spec, _wide(w), 200_000, 12, min_hits=5)
    # every order reflects: rays of 8 / 16 / 24 keV in the three orders' Bragg ranges
    assert t["exit_front"] > 20


def test_fp32_orders_follow_fp64_flat_mixture(H):
    # flat HOPG, a line set for order 1 at 8 keV and one for order 2 (16 keV), plus a
    # continuum: order 2's rays reach the detector only through order 2
    w = W.flat_hopg_mono()
    spec = dict(w["spec"], orders=[(1, 1.0, 1.0), (2, 0.6, 0.7)])
    src = dict(w["source"], components=[dict(kind="gauss", e0_keV=8.0, width_keV=0.004, weight=0.4),
                                        dict(kind="gauss", e0_keV=16.0, width_keV=0.008, weight=0.4),
                                        dict(kind="uniform", lo_keV=7.0, hi_keV=17.0, weight=0.2)])
    r64, r32, t = _fp32_vs_fp64(H, spec, src, 200_000, 13)
    hi = (r32["energy_keV"] > 12.0) & (r32["det_hit"] == 1)
    assert hi.sum() > 5


def test_fp32_single_order_with_multiple_follows_fp64(H):
    # one order given as (m, K ratio, width ratio) = (2, 4, 0.5): sin aB on d / 2, K and
    # the rocking curve of that order, on the FP32 two-pass trace and its records
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], orders=[(2, 4.0, 0.5)], refl_K_per_mm2=5.5e8)
    src = dict(w["source"], components=[dict(kind="gauss", e0_keV=16.0, width_keV=0.02, weight=1.0)])
    _fp32_vs_fp64(H, spec, src, 200_000, 14, min_hits=20)
    import torch
    s = H.heart_spectrometer_create(spec)
    imgs = []
    for prec in ("fp64", "fp32"):
        img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
        H.heart_trace(s, src, 1_000_000, 15, 0, img, precision=prec)
        imgs.append(img.cpu().numpy().astype(np.int64))
    s.close()
    assert imgs[0].sum() > 200
    assert np.abs(imgs[0] - imgs[1]).sum() <= 2e-3 * imgs[0].sum() + 4


def test_fp32_orders_no_rocking_curve_and_polarised(H):
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], orders=ORDERS, irc="none", mdf="gaussian", mdf_fwhm_rad=0.05,
                refl_K_per_mm2=5e9)
    src = dict(_wide(w), polarization=[0.3, 0.9, -0.2])
    _fp32_vs_fp64(H, spec, src, 150_000, 16, min_hits=5)


C_NAMES = dict(ox="origin_x", oy="origin_y", oz="origin_z", kx="dir_x", ky="dir_y", kz="dir_z",
               E="energy_keV", px="pol_x", py="pol_y", pz="pol_z")


@pytest.mark.parametrize("polarised", [False, True])
def test_fp32_orders_user_rays(H, polarised):
    # user rays over 7.5-16.5 keV (orders 1 and 2 in range), entered in FP64 per order
    import torch
    w = W.von_hamos_hapg()
    w = dict(w, source=_wide(w))
    spec = dict(w["spec"], orders=ORDERS)
    n = 200_000
    rays = W.user_rays(w, n, seed=33, polarised=polarised, e_sigma_keV=2.5)
    rays = {C_NAMES[k]: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    s = H.heart_spectrometer_create(spec)
    r64, t64 = H.heart_trace_rays(s, rays, 10, 0, None, precision="fp64", records=True)
    r32, t32 = H.heart_trace_rays(s, rays, 10, 0, None, precision="fp32", records=True)
    s.close()
    flip = (r64["outcome"] != r32["outcome"]) | (r64["nrefl"] != r32["nrefl"]) | (r64["ncoll"] != r32["ncoll"])
    assert flip.sum() <= max(2, 1e-4 * n), int(flip.sum())
    same = ~flip & (r64["det_hit"] == 1) & (r32["det_hit"] == 1)
    assert same.sum() > 5
    assert np.abs(r64["u_mm"][same] - r32["u_mm"][same]).max() <= 1e-3
    assert t32["miss"] == t64["miss"] and t32["no_bragg"] == t64["no_bragg"]


def test_fp32_orders_batch_and_server_equal_single(H):
    # several orders on the two-pass trace (single traces, batch and served jobs of
    # >= 2^18 rays) and on the persistent kernel (static batch, records): the two
    # kernels trace the same rays up to rare rounding-level flips
    import torch
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], orders=ORDERS, irc_energy=TABLE)
    src = _wide(w)
    n = 1 << 22
    s = H.heart_spectrometer_create(spec)
    s2 = H.heart_spectrometer_create(W.flat_hopg_mono()["spec"])
    one = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    t1 = H.heart_trace(s, src, n, 21, 0, one, precision="fp32")
    assert t1["emitted"] == n and t1["det_hits"] == int(one.sum()) > 20
    imgs = [torch.zeros(x.shape, dtype=torch.int32, device="cuda") for x in (s, s2)]
    tb = H.heart_trace_batch([s, s2], [src, W.flat_hopg_mono()["source"]], [n, 100_000], [21, 22], imgs)
    assert torch.equal(one, imgs[0]) and tb[0] == t1
    srv = H.Server(1 << 28)
    jid = srv.submit(s, src, n, 21, precision="fp32")
    _, t, _ = srv.poll(jid, timeout_ms=60_000)
    simg = torch.zeros_like(one)
    srv.fetch(jid, simg)
    srv.release(jid)
    srv.close()
    assert torch.equal(simg, one) and t == t1
    lim = 2 + 1e-4 * n
    stat = [torch.zeros_like(one)]
    ts = H.heart_trace_batch_static([s], [src], [n], [21], stat)
    assert int((stat[0].long() - one.long()).abs().sum()) <= 2 * lim
    assert abs(ts[0]["det_hits"] - t1["det_hits"]) <= lim
    rimg = torch.zeros_like(one)
    _, tr = H.heart_trace_records(s, src, 200_000, 21, 0, precision="fp32", d_image=rimg)
    part = torch.zeros_like(one)
    H.heart_trace(s, src, 200_000, 21, 0, part, precision="fp32")
    assert int((rimg.long() - part.long()).abs().sum()) <= 2 * (2 + 1e-4 * 200_000)
    s.close()
    s2.close()


def test_fp32_no_bragg_cylinder_follows_fp64(H):
    # below the cutoff energy (lambda > 2d) no order reflects: a transparent crystal
    # (constant absorption length) sends rays out of its back face, the exit distance
    # on the cylinder taken from |k.N|
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], absorption_power=0.0, absorption_length_mm=0.5)
    src = dict(w["source"], components=[dict(kind="uniform", lo_keV=1.0, hi_keV=1.8, weight=1.0)])
    s = H.heart_spectrometer_create(spec)
    r64, t64 = H.heart_trace_records(s, src, 100_000, 23, 0, precision="fp64")
    r32, t32 = H.heart_trace_records(s, src, 100_000, 23, 0, precision="fp32")
    s.close()
    assert t64["no_bragg"] == t32["no_bragg"] > 1000
    assert t64["exit_back"] > 100
    flip = r64["outcome"] != r32["outcome"]
    assert flip.sum() <= 2, int(flip.sum())
    out = ~flip & (r64["outcome"] >= 2) & (r64["outcome"] <= 4)      # exits: front, back, side
    assert out.sum() > 100
    assert np.abs(r64["pos"][out] - r32["pos"][out]).max() <= 1e-3
