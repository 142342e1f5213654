"""Pins of the Z-order codes and the radix tree used for the BVH (Sec. 3.3).

* Z-order locality: two cells share the top k bits of every coordinate iff
  their codes share the top 3k bits (the defining property of interleaving);
  the code is a bijection on cells.
* quantisation: the float32 cells agree with exact (FP64) quantisation
  except within float32 rounding of a cell boundary; extremes map to 0/B-1.
* the radix tree equals the branching nodes of a bitwise (Patricia) trie built
  by inserting the augmented keys one by one -- an independent construction.
"""
import numpy as np
import pytest

from oracle import lbvh, morton


def test_interleave_locality_and_bijection():
    rng = np.random.default_rng(0)
    for bits in (10, 21):
        cells = rng.integers(0, 1 << bits, size=(4000, 3)).astype(np.uint64)
        codes = morton.interleave(cells, bits)
        assert len(np.unique(codes)) == len(np.unique(cells, axis=0))
        assert int(codes.max()) < (1 << (3 * bits))
        for _ in range(2000):
            i, j = rng.integers(0, len(cells), size=2)
            # shared top bits of every coordinate
            k = bits
            for a in range(3):
                x = int(cells[i, a]) ^ int(cells[j, a])
                k = min(k, bits - x.bit_length())
            c = int(codes[i]) ^ int(codes[j])
            shared = 3 * bits - c.bit_length()
            assert shared // 3 == k


def test_interleave_bit_order_by_hand():
    """Bit order of the interleave (reading R17): within each 3-bit group x is
    the most significant, then y, then z, lowest group from bit 0.  Codes
    worked out by hand: (1,0,0) -> 0b100, (0,1,0) -> 0b010, (0,0,1) -> 0b001,
    (2,0,0) -> 0b100000, (3,1,2) -> x=11 y=01 z=10 -> groups (x1 y1 z1)(x0 y0 z0)
    = (1 0 1)(1 1 0) = 0b101110, and the top cell (2^b - 1 on every axis) ->
    3b ones."""
    for bits in (10, 21):
        cells = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [3, 1, 2],
                          [(1 << bits) - 1] * 3], dtype=np.uint64)
        want = [0b100, 0b010, 0b001, 0b100000, 0b101110, (1 << (3 * bits)) - 1]
        assert [int(c) for c in morton.interleave(cells, bits)] == want


def test_order_is_stable_and_exact_on_63_bit_codes():
    """order() sorts by (code, original index) (reading R13): equal codes keep
    their input order, and 63-bit codes compare as exact integers (checked
    against Python's integer sort of (code, index) pairs)."""
    rng = np.random.default_rng(5)
    base = rng.normal(size=(300, 3)).astype(np.float32)
    means = base[rng.integers(0, 300, size=2000)]  # many exact duplicates -> equal codes
    for wide in (False, True):
        c, perm = morton.order(means, wide)
        raw = morton.codes(means, wide)
        want = sorted(range(len(raw)), key=lambda i: (int(raw[i]), i))
        assert perm.tolist() == want
        assert [int(x) for x in c] == [int(raw[i]) for i in want]
    # distinct 63-bit codes closer together than float64 can tell apart
    m = np.zeros((3, 3), dtype=np.float32)
    m[:, 0] = [1.0, np.nextafter(np.float32(1.0), np.float32(0.0)), 0.0]
    m[2, 1] = 1.0
    c, perm = morton.order(m, True)
    assert all(int(c[i]) <= int(c[i + 1]) for i in range(len(c) - 1))


def test_quantisation_matches_exact_except_at_boundaries():
    rng = np.random.default_rng(1)
    m = rng.normal(size=(20000, 3)).astype(np.float32)
    for bits in (10, 21):
        cells = morton.quantise(m, bits).astype(np.int64)
        md = m.astype(np.float64)
        lo, hi = md.min(0), md.max(0)
        exact = (md - lo) / (hi - lo) * (1 << bits)
        ref = np.clip(np.floor(exact), 0, (1 << bits) - 1)
        diff = cells - ref
        assert np.all(np.abs(diff) <= 1)
        frac = np.abs(exact - np.round(exact))
        # float32 rounding of v (< 2^bits) is ~2^(bits-24): only cells within that of a boundary move
        tol = 4.0 * 2.0 ** (bits - 24)
        assert np.all((diff == 0) | (frac < tol))
        assert (diff != 0).mean() < 10 * tol
        assert cells.min(0).tolist() == [0, 0, 0]
        assert cells.max(0).tolist() == [(1 << bits) - 1] * 3


def patricia_ranges(keys):
    """Branching nodes of a bitwise trie over augmented keys, as (first, last)."""
    n = len(keys)
    width = 64 + 32
    aug = [(int(k) << 32) | i for i, k in enumerate(keys)]
    root = {}
    for i, a in enumerate(aug):
        node = root
        for b in range(width - 1, -1, -1):
            bit = (a >> b) & 1
            node = node.setdefault(bit, {})
        node["leaf"] = i
    out = set()

    def walk(node):
        if "leaf" in node:
            return node["leaf"], node["leaf"]
        kids = [walk(node[b]) for b in (0, 1) if b in node]
        lo, hi = min(k[0] for k in kids), max(k[1] for k in kids)
        if len(kids) == 2:
            out.add((lo, hi))
        return lo, hi

    walk(root)
    return out


@pytest.mark.parametrize("n,dup", [(2, False), (7, False), (64, False), (300, True)])
def test_radix_tree_equals_patricia_trie(n, dup):
    rng = np.random.default_rng(n)
    hi = 8 if dup else (1 << 30)
    keys = np.sort(rng.integers(0, hi, size=n).astype(np.uint64))
    first, last, split = lbvh.radix_tree(keys)
    assert set(zip(first.tolist(), last.tolist())) == patricia_ranges(keys)
    # children cover the parent's range; each leaf / internal node used once
    leaf_seen = np.zeros(n, int)
    int_seen = np.zeros(n - 1, int)
    int_seen[0] += 1
    for i in range(n - 1):
        a, b, g = first[i], last[i], split[i]
        assert a <= g < b
        assert i in (a, b)
        if g == a:
            leaf_seen[g] += 1
        else:
            assert first[g] == a and last[g] == g
            int_seen[g] += 1
        if g + 1 == b:
            leaf_seen[g + 1] += 1
        else:
            assert first[g + 1] == g + 1 and last[g + 1] == b
            int_seen[g + 1] += 1
    assert np.all(leaf_seen == 1) and np.all(int_seen == 1)
