"""Histogram matching of CT slices (Sec. 3, "Ultrasound simulation": the
learned simulator's input CT slices are matched in intensity histogram to a
subset of its training CT images, to narrow the domain gap).

TEST INFRASTRUCTURE ONLY: used by ``tests/``; never by the product path.

The paper names the operation without fixing its discretisation.  This is
the discrete histogram specification of the image-processing textbooks
(Gonzalez & Woods, "histogram matching"), written so that every decision is
exact:

* bins of width w from h0: bin k(v) = clamp(floor((v - h0) / w), 0, nb - 1),
  the subtraction and division in IEEE FP32;
* S[k] = number of the image's considered pixels in bins 0..k, n = S[nb-1];
  R[m] = the reference's cumulative counts, N = R[nb-1];
* bin k maps to the first reference bin m with R[m] / N >= S[k] / n,
  compared as integers: R[m] n >= S[k] N;
* a considered pixel of bin k becomes that bin's centre h0 + (m + 1/2) w
  (FP32: (m + 0.5) * w, then + h0, each rounded once); other pixels keep
  their value, and an image with no considered pixel is unchanged.
"""
from __future__ import annotations

import numpy as np


def bin_index(v, h0, w, nb):
    """bin of each value (FP32 arithmetic, clamped to the nb bins)"""
    v = np.asarray(v, np.float32)
    q = np.floor((v - np.float32(h0)) / np.float32(w))
    return np.clip(q, 0, nb - 1).astype(np.int64)


def reference_cumulative(values, h0, w, nb):
    """cumulative bin counts R of a set of reference CT values"""
    k = bin_index(np.ravel(values), h0, w, nb)
    return np.cumsum(np.bincount(k, minlength=nb)).astype(np.int64)


def bin_map(S, R):
    """M[k] = first m with R[m] * n >= S[k] * N"""
    S = np.asarray(S, np.int64)
    R = np.asarray(R, np.int64)
    n, N = int(S[-1]), int(R[-1])
    return np.searchsorted(R * n, S * N, side="left").astype(np.int64)


def match(hu, mask, ref_cum, h0, w):
    """one image: hu (float32 [n_pix]), mask (bool [n_pix] or None),
    ref_cum (int64 [nb]) -> matched float32 [n_pix]"""
    hu = np.asarray(hu, np.float32)
    nb = len(ref_cum)
    sel = np.ones(hu.shape, bool) if mask is None else np.asarray(mask, bool)
    out = hu.copy()
    if not sel.any():
        return out
    k = bin_index(hu, h0, w, nb)
    S = np.cumsum(np.bincount(k[sel], minlength=nb)).astype(np.int64)
    M = bin_map(S, ref_cum)
    centre = (M.astype(np.float32) + np.float32(0.5)) * np.float32(w) + np.float32(h0)
    out[sel] = centre[k[sel]]
    return out
