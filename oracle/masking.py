"""Crowded-flavor masking (Sec. 3.1): the pixels affected by saturated sources.

TEST INFRASTRUCTURE ONLY (see the package header).

A pixel is masked (0) when R or S reaches its saturation level anywhere
within a square of half-width `grow` around it (Chebyshev distance, clipped
at the image edges), or when an optional input mask already masks it;
otherwise it is kept (1).  Written as plain loops over the window offsets.
"""
import numpy as np


def saturation_mask(R, S, sat_ref, sat_sci, grow, mask_in=None):
    R = np.asarray(R, np.float64)
    S = np.asarray(S, np.float64)
    n0, n1 = R.shape
    sat = (R >= sat_ref) | (S >= sat_sci)
    hit = np.zeros((n0, n1), dtype=bool)
    for dx in range(-grow, grow + 1):
        for dy in range(-grow, grow + 1):
            # hit[x, y] |= sat[x + dx, y + dy] where that pixel exists
            x0, x1 = max(0, -dx), min(n0, n0 - dx)
            y0, y1 = max(0, -dy), min(n1, n1 - dy)
            if x0 < x1 and y0 < y1:
                hit[x0:x1, y0:y1] |= sat[x0 + dx:x1 + dx, y0 + dy:y1 + dy]
    keep = ~hit
    if mask_in is not None:
        keep &= np.asarray(mask_in) != 0
    return keep.astype(np.uint8)
