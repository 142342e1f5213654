"""Z-order (Morton) codes of Gaussian means -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3.3 (memory reordering of the Gaussians): the mean of each Gaussian is
normalised to the scene box and quantised to integer cells whose bits are
interleaved into a Z-order index; Gaussians are sorted by it.  The quantisation is a floating-point decision that produces an integer,
so it is taken here in the same precision as the kernel (IEEE float32, each
operation rounded to nearest, no fused multiply-add):

    lo, hi  = per-axis min / max of the means            (exact)
    ext     = fl32(hi - lo)
    scale   = fl32(B / ext)          B = 2^10 (30-bit) or 2^21 (63-bit codes)
    v       = fl32(fl32(mu - lo) * scale)
    cell    = min(floor(v), B - 1)

and the code interleaves the cell bits with x most significant:
bit 3i+2 <- x_i, bit 3i+1 <- y_i, bit 3i <- z_i.
"""
from __future__ import annotations

import numpy as np


def quantise(means: np.ndarray, bits: int) -> np.ndarray:
    m = np.ascontiguousarray(np.asarray(means, dtype=np.float32)).reshape(-1, 3)
    B = np.float32(1 << bits)
    if m.shape[0] == 0:
        return np.zeros((0, 3), dtype=np.uint64)
    lo = m.min(axis=0)
    hi = m.max(axis=0)
    ext = (hi - lo).astype(np.float32)
    with np.errstate(divide="ignore"):
        scale = np.where(ext > 0, B / np.where(ext > 0, ext, np.float32(1)), np.float32(0)).astype(np.float32)
    v = ((m - lo).astype(np.float32) * scale).astype(np.float32)
    cell = np.floor(v).astype(np.int64)
    cell = np.clip(cell, 0, (1 << bits) - 1)
    return cell.astype(np.uint64)


def interleave(cells: np.ndarray, bits: int) -> np.ndarray:
    """Bit-interleave integer cells (x most significant)."""
    cells = np.asarray(cells, dtype=np.uint64).reshape(-1, 3)
    code = np.zeros(cells.shape[0], dtype=np.uint64)
    for i in range(bits):
        for axis, off in ((0, 2), (1, 1), (2, 0)):
            bit = (cells[:, axis] >> np.uint64(i)) & np.uint64(1)
            code |= bit << np.uint64(3 * i + off)
    return code


def codes(means: np.ndarray, wide: bool = False) -> np.ndarray:
    bits = 21 if wide else 10
    return interleave(quantise(means, bits), bits)


def order(means: np.ndarray, wide: bool = False):
    """(sorted codes, permutation): stable sort by (code, original index)."""
    c = codes(means, wide)
    perm = np.argsort(c, kind="stable").astype(np.int64)
    return c[perm], perm
