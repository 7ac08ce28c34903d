"""The FP32 kernels (the two-pass trace the benchmark times, which also
writes per-ray records on request, and the persistent kernel of batches)
against the FP64 kernel on the same Philox streams, against each other, and
against an independent-stream oracle image.

Tolerances (fixed before measuring):
  * decision flips (outcome, reflection count or tentative-collision count
    differs: a ray that reflects at another collision took another decision
    even when its outcome and reflection count agree) <= 1e-4 of rays;
  * for rays with the same decisions, detector hit positions within 1 um;
  * line centroid and FWHM of the dispersive profile within 0.1 % of FP64;
  * two-sample chi-square over detector pixels (adjacent pixels of a row
    pooled until the oracle's expected count is >= 5) of the FP32 image
    against an oracle image traced with another seed, with the thinned and
    with the plain sampler: p > 0.01;
  * two FP32 kernels on the same streams: identical images and tallies.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W
from tests.stats_helpers import pixel_chi2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16955_gb300 as H
    return H


def _pair(H, spec, src, n, seed, offset=0):
    s = H.heart_spectrometer_create(spec)
    r64, t64 = H.heart_trace_records(s, src, n, seed, offset, precision="fp64")
    r32, t32 = H.heart_trace_records(s, src, n, seed, offset, precision="fp32")
    s.close()
    return r64, t64, r32, t32


def assert_same_trace(ta, tb, ia, ib):
    """Two FP32 kernels that trace the same streams: every FP32 kernel runs the same
    device functions, compiled without contracting a * b + c beyond the fused
    multiply-adds the source writes out, so each ray takes the same decisions in
    both and images and tallies are identical."""
    import torch
    assert ta == tb, {k: (ta[k], tb[k]) for k in ta if ta[k] != tb[k]}
    assert torch.equal(ia, ib), int((ia.long() - ib.long()).abs().sum())


def _profile_stats(u):
    """centroid and FWHM of a 1-D hit profile (histogram at 1/4 of its rms)"""
    c = float(np.mean(u))
    h, e = np.histogram(u, bins=200, range=(c - 4 * u.std(), c + 4 * u.std()))
    m = h.max()
    above = np.flatnonzero(h >= 0.5 * m)
    fw = e[above[-1] + 1] - e[above[0]]
    return c, fw


@pytest.mark.parametrize("name,n", [("flat_hopg_mono", 200_000), ("von_hamos_hapg", 200_000)])
def test_fp32_same_stream_against_fp64(H, name, n):
    w = getattr(W, name)()
    r64, t64, r32, t32 = _pair(H, w["spec"], w["source"], n, w["seed"])
    assert np.array_equal(r64["ray_id"], r32["ray_id"])
    flip = (r64["outcome"] != r32["outcome"]) | (r64["nrefl"] != r32["nrefl"]) | (r64["ncoll"] != r32["ncoll"])
    assert flip.mean() <= 1e-4, (int(flip.sum()), n)
    same = ~flip & (r64["det_hit"] == 1) & (r32["det_hit"] == 1)
    assert same.sum() > 100
    du = np.abs(r64["u_mm"][same] - r32["u_mm"][same])
    dv = np.abs(r64["v_mm"][same] - r32["v_mm"][same])
    assert du.max() <= 1e-3 and dv.max() <= 1e-3, (du.max(), dv.max())
    # centroid and FWHM of the dispersive profile (detector u), 0.1 %
    u64 = r64["u_mm"][r64["det_hit"] == 1]
    u32 = r32["u_mm"][r32["det_hit"] == 1]
    c64, f64 = _profile_stats(u64)
    c32, f32 = _profile_stats(u32)
    px = w["spec"]["pixel_mm"]
    assert abs(c32 - c64) <= 1e-3 * max(abs(c64), 0.5 * w["spec"]["det_nx"] * px)
    assert abs(f32 - f64) <= 1e-3 * f64 + 1e-9
    # tallies of the same streams agree up to the flipped rays
    assert t32["emitted"] == t64["emitted"]
    assert abs(t32["miss"] - t64["miss"]) <= int(((r64["outcome"] == 0) != (r32["outcome"] == 0)).sum())
    assert abs(t32["det_hits"] - t64["det_hits"]) <= int(flip.sum())
    assert abs(t32["collisions"] - t64["collisions"]) <= 1e-4 * t64["collisions"] + 100 * flip.sum()


@pytest.mark.parametrize("name,n_gpu,n_orc", [("flat_hopg_mono", 8_000_000, 2_000_000),
                                              ("von_hamos_hapg", 20_000_000, 2_000_000)])
def test_fp32_image_matches_independent_oracle(H, name, n_gpu, n_orc):
    import torch
    w = getattr(W, name)()
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    H.heart_trace(s, w["source"], n_gpu, 1002, 0, img, precision="fp32")
    g = img.cpu().numpy().astype(np.int64)
    s.close()
    o, _, _ = ob.trace(w["spec"], w["source"], n_orc, 2002)
    p, pools = pixel_chi2(g, o)
    assert pools >= 50 and p > 0.01, (p, pools)
    # hit fraction
    pg, po = g.sum() / n_gpu, o.sum() / n_orc
    sd = math.sqrt(po * (1 - po) / n_orc + pg * (1 - pg) / n_gpu)
    assert abs(pg - po) <= 4.5 * sd


@pytest.mark.parametrize("name,n_gpu,n_orc", [("flat_hopg_mono", 8_000_000, 2_000_000),
                                              ("von_hamos_hapg", 20_000_000, 2_000_000),
                                              ("von_hamos_large", 20_000_000, 2_000_000)])
def test_fp32_thinned_image_matches_plain_oracle(H, name, n_gpu, n_orc):
    # The FP32 kernels' thinned sampler (process (b) in two tilt bands) against the oracle's
    # plain constant-majorant walk, which draws every candidate and shares none of the
    # thinning: the same image distribution (pixel chi-square) and hit fraction
    import torch
    w = getattr(W, name)()
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int64 if s.count_dtype == "int64" else torch.int32, device="cuda")
    H.heart_trace(s, w["source"], n_gpu, 3003, 0, img, precision="fp32")
    g = img.cpu().numpy().astype(np.int64)
    s.close()
    o, _, _ = ob.trace(dict(w["spec"], sampler="plain"), w["source"], n_orc, 4004)
    p, pools = pixel_chi2(g, o)
    assert pools >= 50 and p > 0.01, (p, pools)
    pg, po = g.sum() / n_gpu, o.sum() / n_orc
    sd = math.sqrt(po * (1 - po) / n_orc + pg * (1 - pg) / n_gpu)
    assert abs(pg - po) <= 4.5 * sd, (pg, po, sd)


def test_fp32_int64_image_and_chunking_invariance(H):
    import torch
    w = W.von_hamos_hapg()
    spec = dict(w["spec"])
    spec["count_type"] = "i64"
    s = H.heart_spectrometer_create(spec)
    a = torch.zeros(s.shape, dtype=torch.int64, device="cuda")
    ta = H.heart_trace(s, w["source"], 1_000_000, 5, 0, a, precision="fp32")
    b = torch.zeros(s.shape, dtype=torch.int64, device="cuda")
    tb1 = H.heart_trace(s, w["source"], 400_000, 5, 0, b, precision="fp32")
    tb2 = H.heart_trace(s, w["source"], 600_000, 5, 400_000, b, precision="fp32")
    s.close()
    # counter-based streams: the image does not depend on how rays are chunked
    assert torch.equal(a, b)
    assert ta["det_hits"] == tb1["det_hits"] + tb2["det_hits"] == int(a.sum())
    assert ta["emitted"] == 1_000_000
    assert ta["emitted"] == (ta["miss"] + ta["absorbed"] + ta["exit_front"] + ta["exit_back"] +
                             ta["exit_side"] + ta["capped"] + ta["stuck"])


def test_fp32_empty_single_ray_and_ragged_traces(H):
    # the two-pass trace at its edges: no rays, one ray, ray counts that leave a ragged
    # last spawn block (257, 4097: one and 16 blocks of 256 plus one ray), and a range
    # of ray ids that crosses 2^32 (the counter's high word), ray by ray against FP64
    import torch
    w = W.von_hamos_hapg()
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    t = H.heart_trace(s, w["source"], 0, 3, 0, img, precision="fp32")
    assert t["emitted"] == 0 and t["det_hits"] == 0 and int(img.abs().sum()) == 0
    for n, off in ((1, 0), (1, 12345), (257, 0), (4097, 0), (4097, (1 << 32) - 2000)):
        r64, t64 = H.heart_trace_records(s, w["source"], n, 3, off, precision="fp64")
        r32, t32 = H.heart_trace_records(s, w["source"], n, 3, off, precision="fp32")
        assert np.array_equal(r32["ray_id"], np.arange(off, off + n, dtype=np.uint64))
        assert t32["emitted"] == n == (t32["miss"] + t32["absorbed"] + t32["exit_front"] + t32["exit_back"] +
                                        t32["exit_side"] + t32["capped"] + t32["stuck"])
        flip = (r64["outcome"] != r32["outcome"]) | (r64["nrefl"] != r32["nrefl"]) | (r64["ncoll"] != r32["ncoll"])
        assert flip.sum() <= 1, (n, off, int(flip.sum()))
        same = ~flip & (r64["det_hit"] == 1) & (r32["det_hit"] == 1)
        if same.any():
            assert np.abs(r64["u_mm"][same] - r32["u_mm"][same]).max() <= 1e-3
        # the image path of the same rays bins exactly the records' hits
        img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
        ti = H.heart_trace(s, w["source"], n, 3, off, img, precision="fp32")
        assert ti == t32 and int(img.sum()) == int((r32["det_hit"] == 1).sum())
    s.close()


def test_multi_chunk_trace_on_two_streams_equals_single_chunk_calls(H):
    # a trace of more than one hit-queue chunk alternates between the queue's two buffers
    # and between the caller's stream and the library's side stream; the same rays traced
    # one chunk per call (one buffer, one stream) give the same image and tallies, on the
    # default stream and on a stream of the caller's
    import torch
    w = W.von_hamos_hapg()
    s = H.heart_spectrometer_create(w["spec"])
    chunk = 1 << 26
    n = 3 * chunk + 12_345
    for stream in (None, torch.cuda.Stream()):
        a = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
        ta = H.heart_trace(s, w["source"], n, 9, 0, a, precision="fp32", stream=stream)
        b = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
        parts = []
        for off in range(0, n, chunk):
            parts.append(H.heart_trace(s, w["source"], min(chunk, n - off), 9, off, b, precision="fp32",
                                       stream=stream))
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        for k in ("emitted", "miss", "absorbed", "exit_front", "exit_back", "exit_side", "det_hits", "collisions"):
            assert ta[k] == sum(p[k] for p in parts), k
        assert ta["emitted"] == n and ta["det_hits"] == int(a.sum()) > 1000
    s.close()


def test_two_pass_trace_equals_persistent_kernel_with_invalid_energies(H):
    # A Gaussian line 4 keV wide about 8 keV draws E <= 0 for ~2 % of the rays: such a ray is a
    # miss.  The image trace (two passes: entry, then the energy of the rays that entered, whose
    # invalid ones travel through the queue as dead records) gives the image and tallies of the
    # persistent kernel (the static batch) on the same streams, exactly; the records mark the
    # rays with invalid energies as misses.
    import torch
    w = W.von_hamos_hapg()
    src = dict(w["source"], components=[dict(kind="gauss", e0_keV=8.0, width_keV=4.0, weight=1.0)],
               cone_half_angle_rad=0.03)
    s = H.heart_spectrometer_create(w["spec"])
    n = 3_000_000
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    t2 = H.heart_trace(s, src, n, 17, 0, img, precision="fp32")
    img_p = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    tp = H.heart_trace_batch_static([s], [src], [n], [17], [img_p])[0]
    img_r = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    rec, tr = H.heart_trace_records(s, src, n, 17, 0, precision="fp32", d_image=img_r)
    s.close()
    assert_same_trace(t2, tp, img, img_p)
    assert_same_trace(t2, tr, img, img_r)
    neg = rec["energy_keV"] < 0                          # entered, then drew a negative energy
    assert neg.sum() > 1000 and np.all(rec["outcome"][neg] == 0)
    assert t2["miss"] > int(neg.sum()) and t2["emitted"] == n
    assert int((rec["outcome"] == 0).sum()) == t2["miss"]


@pytest.mark.parametrize("name", ["flat_hopg_mono", "von_hamos_hapg", "von_hamos_large"])
@pytest.mark.parametrize("sampler", ["thinned", "plain"])
def test_two_pass_trace_equals_persistent_kernel(H, name, sampler):
    # the benchmark's two-pass kernels and the persistent kernel of batches trace every ray
    # alike: identical images and tallies on the same streams (several hit-queue chunks)
    import torch
    w = getattr(W, name)()
    spec = dict(w["spec"], sampler=sampler)
    s = H.heart_spectrometer_create(spec)
    n = (1 << 21) + 4321
    a = torch.zeros(s.shape, dtype=torch.int64 if s.count_dtype == "int64" else torch.int32, device="cuda")
    b = torch.zeros_like(a)
    ta = H.heart_trace(s, w["source"], n, 77, 0, a, precision="fp32")
    tb = H.heart_trace_batch_static([s], [w["source"]], [n], [77], [b])[0]
    s.close()
    assert_same_trace(ta, tb, a, b)
    assert ta["det_hits"] > 100


def test_shared_hit_queue_across_handles_and_streams(H):
    # the two-pass trace's hit queue is one per device: traces of different
    # spectrometers enqueued on two streams at once give the images they give alone
    import torch
    wa, wb = W.von_hamos_hapg(), W.flat_hopg_mono()
    sa, sb = H.heart_spectrometer_create(wa["spec"]), H.heart_spectrometer_create(wb["spec"])
    na, nb = 3_000_000, 20_000_000
    alone = []
    for s, w, n in ((sa, wa, na), (sb, wb, nb)):
        img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
        H.heart_trace(s, w["source"], n, 31, 0, img, precision="fp32")
        alone.append(img)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ia = torch.zeros(sa.shape, dtype=torch.int32, device="cuda")
    ib = torch.zeros(sb.shape, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    H.heart_trace(sa, wa["source"], na, 31, 0, ia, precision="fp32", stream=s1, want_tally=False)
    H.heart_trace(sb, wb["source"], nb, 31, 0, ib, precision="fp32", stream=s2, want_tally=False)
    torch.cuda.synchronize()
    sa.close()
    sb.close()
    assert torch.equal(ia, alone[0]) and torch.equal(ib, alone[1])
    assert int(ia.sum()) > 100 and int(ib.sum()) > 100
