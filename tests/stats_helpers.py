"""Statistics shared by the tests (no part of the ray path)."""
import math

import numpy as np
from scipy import stats


def pixel_chi2(a, b, min_expected=5.0):
    """Two-sample chi-square of two images over pixels: the pixels of each row are
    pooled left to right (adjacent pixels) until the pool's expected count in the
    smaller sample reaches min_expected; a row's remainder joins the last pool
    formed so far.  Returns (p, pools)."""
    A, B = float(a.sum()), float(b.sum())
    small = min(A, B) / (A + B)
    pa, pb = [], []
    ca = cb = 0.0
    for ra, rb in zip(a, b):
        for x, y in zip(ra, rb):
            ca += x
            cb += y
            if (ca + cb) * small >= min_expected:
                pa.append(ca)
                pb.append(cb)
                ca = cb = 0.0
        if ca + cb > 0 and pa:
            pa[-1] += ca
            pb[-1] += cb
            ca = cb = 0.0
    if ca + cb > 0 and pa:
        pa[-1] += ca
        pb[-1] += cb
    pa, pb = np.array(pa), np.array(pb)
    k1, k2 = math.sqrt(B / A), math.sqrt(A / B)
    chi2 = float((((k1 * pa - k2 * pb) ** 2) / (pa + pb)).sum())
    return stats.chi2.sf(chi2, len(pa) - 1), len(pa)
