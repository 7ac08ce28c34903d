"""The tests' own statistics, on synthetic images (CPU)."""
import numpy as np

from tests.stats_helpers import pixel_chi2


def test_pixel_chi2_detects_a_shifted_or_sheared_line():
    # the statistic itself, on synthetic images: equal distributions pass, a line moved
    # by half a pixel or sheared across rows (row sums unchanged) fails
    rng = np.random.default_rng(3)
    yy, xx = np.mgrid[0:64, 0:64]

    def img(shift, shear, n):
        p = np.exp(-0.5 * ((xx - 32 - shift - shear * (yy - 32)) / 2.0) ** 2)
        p /= p.sum()
        return rng.multinomial(n, p.ravel()).reshape(p.shape)

    base, other = img(0, 0, 400_000), img(0, 0, 100_000)
    assert pixel_chi2(base, other)[0] > 0.001
    assert pixel_chi2(base, img(0.5, 0, 100_000))[0] < 1e-6
    assert pixel_chi2(base, img(0, 0.05, 100_000))[0] < 1e-6
