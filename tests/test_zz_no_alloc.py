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
