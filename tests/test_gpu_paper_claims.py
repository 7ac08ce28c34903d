"""A qualitative statement of the paper, checked on the FP32 path.

Sec. 4.3 compares a von Mises-Fisher mosaic distribution with a Gaussian one of
the same FWHM (1 degree) and finds their simulated spectra extremely similar,
as the von Mises-Fisher density tends to the Gaussian for narrow widths
(Sec. 2.2.2).  Here the dispersive line profile of the von Hamos spectrometer
(mono 8 keV source) with the two distributions, on independent streams, must
differ by no more than two independent Gaussian runs differ from each other;
a Lorentzian distribution of the same FWHM, whose tails are much heavier, must
differ clearly."""
import numpy as np
import pytest

from paper_2503_16955_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ONE_DEGREE = 0.017453292519943295


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16955_gb300 as H
    return H


def _profile(H, mdf, seed, n=30_000_000):
    import torch
    w = W.von_hamos_hapg()
    spec = dict(w["spec"], mdf=mdf, mdf_fwhm_rad=ONE_DEGREE)
    src = dict(w["source"], components=[dict(kind="mono", e0_keV=8.0, weight=1.0)])
    s = H.heart_spectrometer_create(spec)
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    H.heart_trace(s, src, n, seed, 0, img)
    s.close()
    return img.sum(dim=0).double().cpu().numpy()          # along the dispersive (axial) direction


def _tv(a, b):
    return 0.5 * np.abs(a / a.sum() - b / b.sum()).sum()


def test_von_mises_fisher_and_gaussian_mosaic_give_the_same_spectrum(H):
    g1, g2 = _profile(H, "gaussian", 5), _profile(H, "gaussian", 6)
    vmf = _profile(H, "vmf", 7)
    lor = _profile(H, "lorentzian", 8)
    assert g1.sum() > 50_000 and vmf.sum() > 50_000 and lor.sum() > 10_000
    noise = _tv(g1, g2)                                    # two independent Gaussian runs
    assert _tv(vmf, g1) < 1.5 * noise + 0.01, (_tv(vmf, g1), noise)
    assert _tv(lor, g1) > 5.0 * noise + 0.1, (_tv(lor, g1), noise)
    x = np.arange(len(g1))
    c = [(p * x).sum() / p.sum() for p in (g1, vmf)]
    assert abs(c[0] - c[1]) < 1.0                          # line centroids within a pixel
