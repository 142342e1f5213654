"""Pins of the oracle's optimiser and densification step.

* Adam: the first step from zero moments moves every entry by lr * g / (|g| + eps)
  (bias correction makes m_hat = g, v_hat = g^2); a run on a convex quadratic
  converges to its minimiser; with the log parameterisation the step equals the
  plain step on log(value) with the chain-ruled gradient (checked by central
  differences of a loss of exp(p)).
* densification: counts and offsets by hand on a small case; clones are exact
  copies; split children with z = 0 sit at the mean with scales s / 1.6, and with
  z = e_j are displaced by s_j times column j of R(q).
"""
import numpy as np

from oracle import train


def test_adam_first_step_and_quadratic():
    rng = np.random.default_rng(0)
    g = rng.normal(size=50)
    p, m, v, _ = train.adam_step(np.zeros(50), g, np.zeros(50), np.zeros(50), lr=0.1, step=1, eps=1e-8)
    np.testing.assert_allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    target = rng.normal(size=8)
    p, m, v = np.zeros(8), np.zeros(8), np.zeros(8)
    for t in range(1, 3001):
        p, m, v, _ = train.adam_step(p, 2 * (p - target), m, v, lr=0.01, step=t)
    assert np.abs(p - target).max() < 1e-3


def test_adam_log_parameterisation_is_the_chain_rule():
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=6)
    c = rng.normal(size=6)

    def loss(p):
        return float((c * np.exp(p) ** 2).sum())

    g_value = 2 * c * np.exp(p0)  # d loss / d value, value = exp(p)
    h = 1e-6
    g_log = np.array([(loss(p0 + h * e) - loss(p0 - h * e)) / (2 * h) for e in np.eye(6)])
    a = train.adam_step(p0, g_value, np.zeros(6), np.zeros(6), lr=0.05, step=3, exp_param=True)
    b = train.adam_step(p0, g_log, np.zeros(6), np.zeros(6), lr=0.05, step=3)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(a[3], np.exp(a[0]))


def test_densify_plan_by_hand():
    stat = np.array([0.0, 3e-4, 1e-4, 9e-4, 5e-4])
    count = np.array([0, 1, 1, 3, 0])
    scales = np.array([[1, 1, 1], [0.01, 0.02, 0.01], [0.5, 0.5, 0.5], [0.2, 0.01, 0.01], [1, 1, 1.0]])
    action, offset, n_out = train.densify_plan(stat, count, scales, tau=1.5e-4, size_threshold=0.05)
    assert action.tolist() == [0, 1, 0, 2, 0]       # 3e-4 > tau small: clone; 1e-4: no; 3e-4 avg, large: split
    assert offset.tolist() == [0, 1, 3, 4, 6] and n_out == 7


def test_densify_apply_clone_and_split_geometry():
    rng = np.random.default_rng(2)
    n = 3
    means, scales = rng.normal(size=(n, 3)), np.exp(rng.normal(-2, 0.3, size=(n, 3)))
    quats, dens = rng.normal(size=(n, 4)), rng.uniform(1, 3, size=n)
    sh = rng.normal(size=(n, 16, 3))
    action = np.array([1, 2, 2], np.int32)
    normals = np.zeros((n, 2, 3))
    normals[2, 1] = [0.0, 1.0, 0.0]
    out = train.densify_apply(action, normals, means, scales, quats, dens, sh)
    assert out["src"].tolist() == [0, 0, 1, 1, 2, 2]
    np.testing.assert_array_equal(out["means"][0], out["means"][1])
    np.testing.assert_array_equal(out["sh"][1], sh[0])
    np.testing.assert_allclose(out["means"][2], means[1])            # z = 0: at the mean
    np.testing.assert_allclose(out["scales"][2], scales[1] / 1.6)
    R = train.rotation(quats[2])
    np.testing.assert_allclose(out["means"][5], means[2] + scales[2, 1] * R[:, 1], rtol=1e-12)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
