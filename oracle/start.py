"""Start values of a fit from the ROI's pixels -- plain reference implementation.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle``): the tests, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU leg may use it; the library never does.

The paper estimates start values from the image before fitting (Results section): a
centre, an amplitude from the extreme pixel values, and a width from the number of pixels
above the level a Gaussian reaches at one sigma, M ~ pi sigma^2, so sigma0 = sqrt(M / pi).
Two centre rules:

* CENTROID  centroid of max(g - b0, 0) with b0 = min g (the ROI centre if the weight is zero
            everywhere; a reading: the paper does not say);
* PAPER     the pixel whose 3 x 3 neighbourhood, clipped to the ROI, has the largest mean;
            ties go to the lowest row-major index (a reading).

Readings that fix the precision of the integer decisions (the same as the kernel's, so that
both sides decide alike): the amplitude a0 = max g - min g, the threshold fl(fl(a0 c) + b0)
with c = e^(-1/2) rounded to FP32 and every product and sum in FP32; a pixel counts in M when
its FP32 value exceeds that threshold; two neighbourhood means are compared as
S_i c_j > S_j c_i with c the neighbour count and S summed in FP32 row by row: each row's
in-ROI neighbours left to right, then those row sums top to bottom; the products in FP32.
For integer-valued pixels below 2^21 all of these are exact. The centroid and sigma0
themselves are computed in FP64 here.

parity unpinned: the zero-weight fallback (ROI centre) and the tie rule of PAPER are
conventions, not the paper's.
"""
from __future__ import annotations

import math

import numpy as np

CENTROID, PAPER = 0, 1
ONE_SIGMA_F32 = np.float32(math.exp(-0.5))


def start_one(g: np.ndarray, W: int, H: int, rule: int) -> np.ndarray:
    """(x0, y0, s0, s0) of one ROI; g holds its W*H pixels row by row."""
    img = np.asarray(g, dtype=np.float32).reshape(H, W)
    b0 = img.min()
    a0 = np.float32(img.max() - b0)
    thr = np.float32(np.float32(a0 * ONE_SIGMA_F32) + b0)
    M = int((img > thr).sum())
    s0 = math.sqrt(max(M, 1) / math.pi)
    if rule == PAPER:
        best = None
        for y in range(H):
            for x in range(W):
                S = np.float32(0.0)
                c = 0
                for dy in (-1, 0, 1):
                    if not 0 <= y + dy < H:
                        continue
                    row = np.float32(0.0)
                    for dx in (-1, 0, 1):
                        if 0 <= x + dx < W:
                            row = np.float32(row + img[y + dy, x + dx])
                            c += 1
                    S = np.float32(S + row)
                if best is None or np.float32(S * np.float32(best[1])) > np.float32(best[0] * np.float32(c)):
                    best = (S, c, x, y)
        x0, y0 = float(best[2]), float(best[3])
    else:
        w = np.maximum(img.astype(np.float64) - float(b0), 0.0)
        sw = w.sum()
        if sw > 0:
            ys, xs = np.mgrid[0:H, 0:W]
            x0 = float((w * xs).sum() / sw)
            y0 = float((w * ys).sum() / sw)
        else:
            x0, y0 = 0.5 * (W - 1), 0.5 * (H - 1)
    return np.array([x0, y0, s0, s0])


def start_values(images: np.ndarray, offsets, dims, rule: int = CENTROID) -> np.ndarray:
    """[n, 4] start values; an ROI outside 1..32 per side or outside the buffer gets NaNs."""
    offsets = np.asarray(offsets, dtype=np.int64)
    dims = np.asarray(dims, dtype=np.int64).reshape(-1, 2)
    out = np.full((offsets.size, 4), np.nan)
    for s in range(offsets.size):
        W, H = int(dims[s, 0]), int(dims[s, 1])
        o = int(offsets[s])
        if not (1 <= W <= 32 and 1 <= H <= 32 and o >= 0 and o + W * H <= images.size):
            continue
        out[s] = start_one(images[o:o + W * H], W, H, rule)
    return out
