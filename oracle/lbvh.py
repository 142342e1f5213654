"""Binary radix tree over sorted Morton codes -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper keeps its Gaussians in a BVH over their AABBs, rebuilt at every
optimisation step (Sec. 3.2, Sec. 3.4).  The GPU builds it as a linear BVH: a
binary radix tree over the Z-order-sorted keys.  The tree is a pure function of
the sorted keys, so it is checked bit for bit against this plain top-down
definition:

* keys are made unique by appending the sorted position (key, i);
* the node covering sorted range [a, b] (a < b) splits after the last
  position whose key has a 0 at the most significant bit where key_a and
  key_b differ;
* node numbering follows the usual linear layout: the root is internal node 0;
  an internal child that is a *left* child takes the index of the last
  position of its range, a *right* child the index of its first position.

Returned arrays, per internal node i in [0, N-1): first[i], last[i], split[i]
(left child covers [first, split], right child [split+1, last]).
"""
from __future__ import annotations

import numpy as np


def radix_tree(sorted_codes: np.ndarray):
    keys = [int(k) for k in np.asarray(sorted_codes, dtype=np.uint64)]
    n = len(keys)
    if n < 2:
        z = np.zeros(0, dtype=np.int64)
        return z, z.copy(), z.copy()
    aug = [(k << 32) | i for i, k in enumerate(keys)]
    first = np.full(n - 1, -1, dtype=np.int64)
    last = np.full(n - 1, -1, dtype=np.int64)
    split = np.full(n - 1, -1, dtype=np.int64)
    stack = [(0, n - 1, 0)]  # (a, b, node index)
    while stack:
        a, b, node = stack.pop()
        top = (aug[a] ^ aug[b]).bit_length() - 1
        # last position in [a, b-1] whose bit `top` is 0 (keys are sorted)
        lo, hi = a, b
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if (aug[mid] >> top) & 1:
                hi = mid
            else:
                lo = mid
        g = lo
        first[node], last[node], split[node] = a, b, g
        if g > a:
            stack.append((a, g, g))
        if g + 1 < b:
            stack.append((g + 1, b, g + 1))
    return first, last, split
