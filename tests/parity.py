"""Error measures of the parity tests (CUDA path against the oracle).

elem_rel(a, b): the largest element-by-element relative difference
|a_k - b_k| / (|b_k| + FLOOR * max_j |b_j|).  Entries at least FLOOR (1e-3)
of the array's largest magnitude are compared in relative terms; smaller
ones are differences of larger numbers, whose FP64 round-off is set by the
array's scale, so they are held to the floor instead.  Used for records,
weights, ratios and Green's functions.

norm_rel(a, b): max_k |a_k - b_k| / max_k |b_k|, for the QR factors of a
stabilization block.  A backward-stable QR (Householder in the oracle,
CholeskyQR2 on the GPU) of a graded panel is accurate relative to the
panel's scale, not entry by entry, so these are compared normwise; the
quantity they feed, log|W| = sum log V_kk + log|det P^T Q|, is compared
entry by entry.
"""
import numpy as np

FLOOR = 1e-3


def elem_rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if a.shape != b.shape:
        return float("inf")
    if b.size == 0:
        return 0.0
    scale = float(np.max(np.abs(b)))
    den = np.abs(b) + FLOOR * scale
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(a - b) / den))


def norm_rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if a.shape != b.shape:
        return float("inf")
    if b.size == 0:
        return 0.0
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0))


def weight_rel(lw_a, lw_b):
    """Relative difference of two log-weights, |a - b| / max(1, |b|)."""
    return abs(lw_a - lw_b) / max(1.0, abs(lw_b))
