"""The CUDA path through the C-ABI on the stored oracle render of the explicit
5-Gaussian scene (tests/golden/tiny_render.json): RGBA within max-abs 1e-4 and
every gradient tensor within 1e-3 relative L2, in both marching modes."""
import json
import os
import sys

import numpy as np
import pytest

from helpers import TOL_GRAD, TOL_RGBA, gpu_backward, gpu_render, rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402


@pytest.mark.parametrize("mode", ["uniform", "adaptive_skip"])
def test_tiny_scene_matches_the_stored_oracle_values(mode):
    with open(os.path.join(GOLDEN, "tiny_render.json")) as f:
        gold = json.load(f)["modes"][mode]
    sc, cam = make_golden.tiny_scene(), make_golden.tiny_camera()
    o = make_golden.modes()[mode]
    r = gpu_render(sc, [cam], o)
    assert r["status"] == 0
    err = np.abs(r["rgba"] - np.array(gold["rgba"])).max()
    assert err <= TOL_RGBA, err
    g = gpu_backward(r, make_golden.upstream(cam.n_rays))
    assert g["status"] == 0
    for k, v in gold["grad"].items():
        e = rel_l2(g[k], np.array(v))
        assert e <= TOL_GRAD, (k, e)
