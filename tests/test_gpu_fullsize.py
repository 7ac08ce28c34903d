"""Full-size workloads in the launch configuration the benchmark times.

* flat HOPG mono (2e5 rays, the whole workload): FP64 kernel vs the oracle,
  ray by ray; FP32 two-pass kernels flip within 1e-4.
* von Hamos HAPG at 1e8 rays (the benchmark's step, FP32, one call: two
  hit-queue chunks of up to 2^26 rays on two streams): the records that this
  launch's spawn and walk kernels write, taken from windows of ray ids spread
  over the range and straddling the chunk boundary, against the FP64 kernel
  and the oracle ray by ray (outcome flips <= 1e-4, hits within 1 um); the
  launch's image and tallies against its own records and an oracle sample.
* large von Hamos job at 1e9 rays into a 4096^2 int64 image (the 1e10-ray
  job streams such launches by ray offset): invariants and sampled windows.
"""
import math

import numpy as np
import pytest

from oracle import binding as ob
from paper_2503_16955_gb300 import workloads as W

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


def _conserved(t):
    return t["emitted"] == (t["miss"] + t["absorbed"] + t["exit_front"] + t["exit_back"] + t["exit_side"] +
                            t["capped"] + t["stuck"])


def _windows(H, spec, w, starts, size, precision):
    for s0 in starts:
        g, _ = H.heart_trace_records(spec, w["source"], size, w["seed"], s0, precision=precision)
        _, _, o = ob.trace(w["spec"], w["source"], size, w["seed"], ray_offset=s0, records=True)
        yield g, o


def test_flat_hopg_full_workload_fp64_and_fp32(H):
    w = W.flat_hopg_mono()
    s = H.heart_spectrometer_create(w["spec"])
    g, gt = H.heart_trace_records(s, w["source"], w["n_rays"], w["seed"], 0, precision="fp64")
    o_img, ot, o = ob.trace(w["spec"], w["source"], w["n_rays"], w["seed"], records=True)
    assert np.array_equal(g["outcome"], o["outcome"]) and np.array_equal(g["nrefl"], o["nrefl"])
    assert np.array_equal(g["ncoll"], o["ncoll"])
    hit = o["det_hit"] == 1
    assert np.all(np.abs(g["u_mm"][hit] - o["u_mm"][hit]) <= 1e-9 * np.maximum(1, np.abs(o["u_mm"][hit])))
    assert gt == ot
    g32, t32 = H.heart_trace_records(s, w["source"], w["n_rays"], w["seed"], 0, precision="fp32")
    flips = ((g32["outcome"] != o["outcome"]) | (g32["nrefl"] != o["nrefl"]) | (g32["ncoll"] != o["ncoll"])).mean()
    assert flips <= 1e-4
    s.close()


def test_von_hamos_benchmark_step_full_size(H):
    import torch
    w = W.von_hamos_hapg()
    n = 100_000_000
    chunk = 1 << 26
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    rec, t = H.heart_trace_records(s, w["source"], n, w["seed"], 0, precision="fp32", d_image=img, on_device=True)
    assert t["emitted"] == n and _conserved(t)
    assert t["det_hits"] == int(img.sum()) and int(img.min()) >= 0
    assert t["stuck"] == 0
    # the same launch without records gives the same image and tallies
    img2 = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    t2 = H.heart_trace(s, w["source"], n, w["seed"], 0, img2, precision="fp32")
    assert torch.equal(img, img2) and t2 == t
    # tallies against an independent oracle sample of 1e6 rays
    _, ot, _ = ob.trace(w["spec"], w["source"], 1_000_000, 4242)
    for k in ("miss", "absorbed", "exit_front", "exit_back", "det_hits"):
        p, q = t[k] / n, ot[k] / 1e6
        sd = math.sqrt(max(q * (1 - q), 1e-12) / 1e6 + max(p * (1 - p), 1e-12) / n)
        assert abs(p - q) <= 5 * sd + 1e-7, (k, p, q)
    # windows of this launch's records, including the chunk boundary, one by one
    flips = total = 0
    for s0, size in ((0, 20_000), (33_000_000, 20_000), (chunk - 10_000, 20_000), (81_000_000, 20_000),
                     (n - 20_000, 20_000)):
        g = H.records_from_device(rec, s0, size)
        f64, _ = H.heart_trace_records(s, w["source"], size, w["seed"], s0, precision="fp64")
        _, _, o = ob.trace(w["spec"], w["source"], size, w["seed"], ray_offset=s0, records=True)
        assert np.array_equal(g["ray_id"], np.arange(s0, s0 + size, dtype=np.uint64))
        assert np.array_equal(f64["outcome"], o["outcome"]) and np.array_equal(f64["nrefl"], o["nrefl"])
        same = (g["outcome"] == f64["outcome"]) & (g["nrefl"] == f64["nrefl"]) & (g["ncoll"] == f64["ncoll"])
        flips += int((~same).sum())
        total += size
        both = same & (g["det_hit"] == 1) & (f64["det_hit"] == 1)
        assert np.all(np.abs(g["u_mm"][both] - f64["u_mm"][both]) <= 1e-3)
        assert np.all(np.abs(g["v_mm"][both] - f64["v_mm"][both]) <= 1e-3)
        assert both.sum() > 0 or size < 50_000
    assert flips <= max(1, 1e-4 * total), (flips, total)
    # the image is the binning of the launch's records (fields read on the device:
    # ix, iy, det_hit are 32-bit words 24, 25, 26 of a 136-byte record)
    assert H.RECORD_DTYPE.fields["ix"][1] == 96 and H.RECORD_DTYPE.fields["det_hit"][1] == 104
    words = rec.view(torch.int32).view(n, H.RECORD_DTYPE.itemsize // 4)
    hit = words[:, 26] == 1
    pix = (words[:, 25][hit].long() * s.shape[1] + words[:, 24][hit].long())
    binned = torch.bincount(pix, minlength=s.shape[0] * s.shape[1]).view(s.shape)
    assert torch.equal(binned.to(torch.int32), img)
    del words, rec
    s.close()


def test_large_job_int64_image_streamed_chunk(H):
    import torch
    w = W.von_hamos_large()
    n = 1_000_000_000
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int64, device="cuda")
    t = H.heart_trace(s, w["source"], n, w["seed"], 3 * n, img, precision="fp32")
    assert t["emitted"] == n and _conserved(t)
    assert t["det_hits"] == int(img.sum())
    flips = total = 0
    for g, o in _windows(H, s, w, [3 * n, 3 * n + 500_000_000], 5_000, "fp32"):
        flips += int(((g["outcome"] != o["outcome"]) | (g["nrefl"] != o["nrefl"]) | (g["ncoll"] != o["ncoll"])).sum())
        total += len(g)
    assert flips <= max(1, 1e-4 * total)
    s.close()
