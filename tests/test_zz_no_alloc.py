"""The allocation-free Morton sort gives the same codes and permutation as the
BVH build of a scene, on two calls in a row.

rgx_morton_sort_noalloc is for callers that cannot call cudaMalloc (code
running during a CUDA-graph capture, plugins inside an engine that owns all
device memory, loops that must not allocate).  Its scratch is one static
device array shared by every call, so this test also checks that a second
call with different data is not disturbed by what the first one left behind.
Integer outputs: compared bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2509_07782_b300 import rgx, synth

pytestmark = pytest.mark.gpu


def build_codes(scene, wide):
    sc = rgx.Scene()
    t = rgx.scene_tensors(scene)
    sc.build(*t, rgx.make_opts(synth.fast_options(morton63=wide)))
    codes, perm, _, _ = sc.bvh()
    assert sc.status() == 0
    return codes.clone(), perm.clone(), t[0]


@pytest.mark.parametrize("wide", [False, True])
def test_noalloc_sort_matches_build_on_two_calls(wide):
    scenes = [synth.workload("torus_100k", n=50_000).scene, synth.workload("outdoor_3m", n=200_000).scene]
    expected = [build_codes(s, wide) for s in scenes]
    for (codes_ref, perm_ref, means) in expected:
        n = means.shape[0]
        codes = torch.full((n,), -1, dtype=torch.int64, device=means.device)
        perm = torch.full((n,), -1, dtype=torch.int32, device=means.device)
        rgx.rgx_morton_sort_noalloc(means, wide, codes, perm)
        torch.cuda.synchronize()
        assert torch.equal(codes, codes_ref)
        assert torch.equal(perm, perm_ref)


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    n = 262_144 + 1
    means = torch.zeros(n, 3, dtype=torch.float32, device="cuda")
    codes = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(rgx.RgxError) as e:
        rgx.rgx_morton_sort_noalloc(means, False, codes, perm)
    assert e.value.code == rgx.RGX_ERR_INVALID_ARG


@pytest.mark.parametrize("wide", [False, True])
def test_noalloc_sort_at_its_maximum_size_matches_the_oracle_order(wide):
    """n = 262,144 (the whole static region in use, every histogram block
    filled): bit-exact against the oracle's stable sort of its own Z-order
    codes, and against the BVH build."""
    import oracle.morton as om
    scene = synth.workload("torus_100k", n=262_144).scene
    codes_ref, perm_ref, means = build_codes(scene, wide)
    n = means.shape[0]
    assert n == 262_144
    codes = torch.empty(n, dtype=torch.int64, device=means.device)
    perm = torch.empty(n, dtype=torch.int32, device=means.device)
    for _ in range(2):
        codes.fill_(-1)
        perm.fill_(-1)
        rgx.rgx_morton_sort_noalloc(means, wide, codes, perm)
        torch.cuda.synchronize()
        assert torch.equal(codes, codes_ref) and torch.equal(perm, perm_ref)
    oc, op = om.order(scene.means, wide)
    np.testing.assert_array_equal(codes.cpu().numpy().view(np.uint64), oc)
    np.testing.assert_array_equal(perm.cpu().numpy().astype(np.int64), op)


def test_noalloc_sort_allocates_nothing():
    """After its first call on the device (which looks up the array's address),
    a call leaves the device's free memory exactly as it was: nothing is
    allocated, by the library or through the runtime."""
    scene = synth.workload("outdoor_3m", n=150_000).scene
    codes_ref, perm_ref, means = build_codes(scene, True)
    n = means.shape[0]
    codes = torch.empty(n, dtype=torch.int64, device=means.device)
    perm = torch.empty(n, dtype=torch.int32, device=means.device)
    rgx.rgx_morton_sort_noalloc(means, True, codes, perm)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        codes.fill_(0)
        rgx.rgx_morton_sort_noalloc(means, True, codes, perm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(codes, codes_ref) and torch.equal(perm, perm_ref)
