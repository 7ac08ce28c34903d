"""Device functions of the FP32 kernels, evaluated on dense grids through the
C ABI (heart_check_functions) and checked against FP64 references.

* acos_ratio (the arc ends of the thinned sampler's azimuth arcs): Abramowitz
  & Stegun 4.4.46 approximates acos(x) on [0, 1] as sqrt(1 - x) times a
  degree-7 polynomial with |error| <= 2e-8; in FP32 the function forms
  1 - |x| as (b - |m|) / b and multiplies by an approximate reciprocal
  (relative error of 1 - x and of the square root each ~2^-22, of the Horner
  sum ~2^-21), so its error against acos(m / b) is bounded by
  2e-8 + 2^-20 (acos + 1) (under 2.1e-6 rad).
* the rocking curves R / R_max and the bound the kernels' early rejection uses:
  for every rocking curve the bound at |x| is at least R(x') / R_max for every
  |x'| >= |x| (the 1e-5 relative margin covers the approximate reciprocal and
  exponential that form it), and the curve itself matches the FP64 oracle's.
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


def test_acos_ratio_against_fp64_acos(H):
    import torch
    bs = np.array([1e-4, 3e-3, 0.07, 0.5, 1.0], dtype=np.float32)
    for b in bs:
        # m over [-b, b], dense, with extra points next to +-b where sqrt(1 - x) is steepest
        u = np.concatenate([np.linspace(-1.0, 1.0, 400_001), 1.0 - np.geomspace(1e-7, 1e-2, 5000),
                            -1.0 + np.geomspace(1e-7, 1e-2, 5000)])
        m = (u * b).astype(np.float32)
        bb = np.full_like(m, b)
        got = H.heart_check_functions(None, "acos_ratio", torch.from_numpy(m).cuda(),
                                      torch.from_numpy(bb).cuda()).cpu().numpy().astype(np.float64)
        x = np.clip(m.astype(np.float64) / np.float64(b), -1.0, 1.0)
        ref = np.arccos(x)
        bound = 2e-8 + 2.0 ** -20 * (ref + 1.0)
        err = np.abs(got - ref)
        assert np.all(err <= bound), (float(b), float(err.max()), float(u[np.argmax(err - bound)]))
    # beyond the ends: clamped to 0 and pi
    m = torch.tensor([2.0, -2.0, 1.0, -1.0], dtype=torch.float32, device="cuda")
    out = H.heart_check_functions(None, "acos_ratio", m, torch.ones(4, dtype=torch.float32, device="cuda"))
    assert out.cpu().tolist()[:3] == [0.0, pytest.approx(math.pi, abs=1e-6), 0.0]


RC = [("darwin", {}), ("darwin_prins", {"prins_g": 0.05}), ("pseudo_voigt", {"irc_lorentz_fwhm_rad": 8e-6}),
      ("gaussian", {}), ("lorentzian", {}), ("box", {})]


@pytest.mark.parametrize("irc,kw", RC)
def test_rocking_curve_and_its_early_rejection_bound(H, irc, kw):
    import torch
    spec = dict(W.flat_hopg_mono()["spec"], irc=irc, irc_fwhm_rad=20e-6, prins_g=0.0, irc_lorentz_fwhm_rad=0.0)
    spec.update(kw)
    s = H.heart_spectrometer_create(spec)
    a = np.concatenate([np.linspace(0.0, 2e-4, 20_001), np.geomspace(2e-4, 1.0, 4000)]).astype(np.float32)
    ta = torch.from_numpy(a).cuda()
    rel = H.heart_check_functions(s, "irc_rel", ta).cpu().numpy().astype(np.float64)
    bound = H.heart_check_functions(s, "irc_bound", ta).cpu().numpy().astype(np.float64)
    s.close()
    # the bound at a covers the curve everywhere beyond a (suffix maximum on the grid)
    suffix = np.maximum.accumulate(rel[::-1])[::-1]
    assert np.all(bound >= suffix), (irc, float(a[np.argmax(suffix - bound)]), float((suffix - bound).max()))
    # the FP32 curve against the FP64 oracle's, relative to the maximum: the FP32 kernel
    # forms the curve's argument (y = x / delta and the like) to a few ulp, which moves it
    # by the curve's slope times 2^-21 x (a large move at the Darwin plateau's edge, where
    # sqrt(y^2 - 1) has infinite slope), and evaluates it to ~1e-6
    ax = a.astype(np.float64)
    rmax = ob.irc_max(spec)
    ref = ob.irc(spec, ax) / rmax
    lo = ob.irc(spec, ax * (1 - 2.0 ** -21)) / rmax
    hi = ob.irc(spec, ax * (1 + 2.0 ** -21)) / rmax
    tol = np.maximum(np.abs(hi - ref), np.abs(lo - ref)) + 1e-6
    bad = np.abs(rel - ref) > tol
    assert not bad.any(), (irc, float(a[bad][0]), float(rel[bad][0]), float(ref[bad][0]))


def test_arc_bound_lies_above_the_thinned_samplers_arc_measure(H):
    # The walk rejects a process-(b) candidate before computing its azimuth arcs when
    # t3 pbar is at least the sum of the two arcs' bounds; the rejection changes no
    # outcome only if each bound lies above the measure arc_sample computes for the
    # arc (by more than the rounding of a two-term sum).  Intervals (lo, hi) / b over
    # [-1.2, 1.2], narrow ones, ones next to +-1 and ones across it, for b over 8 decades.
    import torch
    rng = np.random.default_rng(11)
    for b in (1e-7, 2e-5, 3e-3, 0.07, 0.5, 0.93, 1.0):
        parts = []
        c = rng.uniform(-1.2, 1.2, (2, 300_000))
        parts.append((c.min(0), c.max(0)))
        mid = rng.uniform(-1.0, 1.0, 200_000)
        wid = np.geomspace(1e-7, 1e-1, 200_000)
        parts.append((mid - wid, mid + wid))
        e = np.geomspace(1e-8, 2.0, 700)
        e1, e2 = np.meshgrid(e, e)
        m = e1 > e2
        parts.append((1.0 - e1[m], 1.0 - e2[m]))             # next to +1
        parts.append((-1.0 + e2[m], -1.0 + e1[m]))           # next to -1
        lo = np.concatenate([p[0] for p in parts]) * b
        hi = np.concatenate([p[1] for p in parts]) * b
        x = torch.from_numpy(lo.astype(np.float32)).cuda()
        y = torch.from_numpy(hi.astype(np.float32)).cuda()
        z = torch.full_like(x, b)
        bound = H.heart_check_functions(None, "arc_bound", x, y, z).cpu().numpy().astype(np.float64)
        meas = H.heart_check_functions(None, "arc_measure", x, y, z).cpu().numpy().astype(np.float64)
        lo32, hi32 = x.cpu().numpy(), y.cpu().numpy()
        b32 = np.float32(b)
        empty = ~((lo32 < hi32) & (lo32 < b32) & (hi32 > -b32))   # no arc: both are 0
        assert np.all(bound[empty] == 0.0) and np.all(meas[empty] == 0.0)
        gap = (bound - meas)[~empty]
        assert empty.mean() < 0.2 and np.all(gap >= 1e-6), (b, float(gap.min()))
        # and above the exact measure of the FP32 interval
        c1 = np.clip(lo32.astype(np.float64) / np.float64(b32), -1, 1)
        c2 = np.clip(hi32.astype(np.float64) / np.float64(b32), -1, 1)
        exact = np.where(c1 < c2, np.arccos(c1) - np.arccos(c2), 0.0) / math.pi
        assert np.all(bound >= exact), (b, float((exact - bound).max()))
        # the bound is no trivial one: within a factor 2.3 of the measure (plus its margin)
        assert np.all(bound <= 2.3 * exact + 1e-5), (b, float((bound - 2.3 * exact).max()))
