"""BVH build parity (integer work: bit-exact) and box conservativeness.

* sorted Morton codes and the permutation equal the oracle's float32
  quantisation + stable sort (30- and 63-bit codes), also when many
  Gaussians share a code;
* every internal node's (first, split, last) equals the radix tree of the
  sorted codes;
* every leaf box contains its Gaussian's sigma_eps ellipsoid (oracle FP64
  half-lengths) and every parent box contains its children.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import lbvh, morton
from paper_2509_07782_b300 import rgx, synth

pytestmark = pytest.mark.gpu


def build(scene, opts):
    sc = rgx.Scene()
    t = rgx.scene_tensors(scene)
    sc.build(*t, rgx.make_opts(opts), sh_degree=scene.sh_degree)
    codes, perm, nodes, root = sc.bvh()
    assert sc.status() == 0
    return codes.cpu().numpy().view(np.uint64), perm.cpu().numpy(), nodes.cpu().numpy(), root.cpu().numpy()


@pytest.mark.parametrize("name,n,wide", [("plain_2k", None, False), ("torus_100k", 20000, False),
                                         ("torus_100k", 20000, True), ("outdoor_3m", 50000, True)])
def test_codes_perm_and_tree_bit_exact(name, n, wide):
    w = synth.workload(name, n=n)
    o = synth.fast_options(morton63=wide)
    codes, perm, nodes, root = build(w.scene, o)
    ref_codes, ref_perm = morton.order(w.scene.means, wide=wide)
    np.testing.assert_array_equal(codes, ref_codes)
    np.testing.assert_array_equal(perm, ref_perm)
    first, last, split = lbvh.radix_tree(ref_codes)
    nn = len(first)
    ints = nodes[:nn].view(np.int32)
    np.testing.assert_array_equal(ints[:, 3], first)
    np.testing.assert_array_equal(ints[:, 7], split)
    np.testing.assert_array_equal(ints[:, 11], last)


@pytest.mark.parametrize("wide", [False, True])
def test_equal_codes_keep_index_order_and_split_by_position(wide):
    """Many Gaussians at exactly the same mean share one Morton code: the sort
    must keep them in caller order and the radix tree must split the run of
    equal codes by sorted position, as the oracle's (code, index) keys do."""
    w = synth.workload("plain_2k")
    rng = np.random.default_rng(9)
    pick = rng.integers(0, 300, size=w.scene.n)
    sc = synth.Scene(w.scene.means[pick], w.scene.scales, w.scene.quats, w.scene.densities, w.scene.sh, 3)
    codes, perm, nodes, _ = build(sc, synth.fast_options(morton63=wide))
    ref_codes, ref_perm = morton.order(sc.means, wide=wide)
    assert len(np.unique(ref_codes)) < sc.n // 2
    np.testing.assert_array_equal(codes, ref_codes)
    np.testing.assert_array_equal(perm, ref_perm)
    first, last, split = lbvh.radix_tree(ref_codes)
    ints = nodes[:len(first)].view(np.int32)
    np.testing.assert_array_equal(ints[:, 3], first)
    np.testing.assert_array_equal(ints[:, 7], split)
    np.testing.assert_array_equal(ints[:, 11], last)


def test_boxes_are_conservative():
    w = synth.workload("torus_100k", n=5000)
    o = synth.fast_options()
    codes, perm, nodes, root = build(w.scene, o)
    _, _, Qe, half = oracle.prim_geometry(w.scene, o.sigma_eps)
    mu = w.scene.means.astype(np.float64)
    n = w.scene.n
    ints = nodes.view(np.int32)
    box = np.zeros((2 * n - 1, 6))  # leaves then internal nodes
    for i in range(n - 1):
        first, split, last = ints[i, 3], ints[i, 7], ints[i, 11]
        lbox = np.r_[nodes[i, 0:3], nodes[i, 4:7]]
        rbox = np.r_[nodes[i, 8:11], nodes[i, 12:15]]
        for child, b in ((split, lbox) if first == split else (n + split, lbox),
                         (split + 1, rbox) if split + 1 == last else (n + split + 1, rbox)):
            box[child] = b
    for i in range(n):
        l = perm[i]
        lo, hi = box[i, :3], box[i, 3:]
        assert np.all(lo <= mu[l] - half[l]) and np.all(hi >= mu[l] + half[l])
        assert np.all(hi - lo <= 2 * half[l] * 1.001 + 1e-5)
    for i in range(n - 1):
        nb = box[n + i] if i > 0 else np.r_[root[:3], root[3:]]
        for b in (np.r_[nodes[i, 0:3], nodes[i, 4:7]], np.r_[nodes[i, 8:11], nodes[i, 12:15]]):
            assert np.all(b[:3] >= nb[:3]) and np.all(b[3:] <= nb[3:])


def test_single_and_empty_scene_build():
    w = synth.workload("plain_2k", n=1)
    codes, perm, nodes, root = build(w.scene, w.options)
    assert perm.tolist() == [0]
    w0 = synth.workload("plain_2k", n=1)
    empty = w0.scene.subset(np.zeros(0, dtype=np.int64))
    sc = rgx.Scene()
    t = rgx.scene_tensors(empty)
    sc.build(*t, rgx.make_opts(w0.options))
    assert sc.status() == 0
    torch.cuda.synchronize()
