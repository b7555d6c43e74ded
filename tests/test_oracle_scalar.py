"""Pins of the oracle's scalar operators against their definitions.

* prox_cost: argmin of 0.5 (z - v)^2 + gamma (c1 |z| + c2 |z|^d), the
  per-asset trading cost of Eq. 1 (spread + power impact, d in (1, 2]).
* project_l1: projection onto the budget set of Eq. 3.
* cost_conjugate: Fenchel conjugate of c1 |z| + c2 |z|^d.
"""
import numpy as np
import pytest

from oracle.prox import cost_conjugate, l1_threshold, prox_cost, project_l1


def _golden_min(fun, lo, hi, iters=200):
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = fun(c), fun(d)
    for _ in range(iters):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = fun(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = fun(d)
    return 0.5 * (a + b)


@pytest.mark.parametrize("d", [1.1, 1.5, 2.0])
def test_prox_matches_direct_minimisation(d):
    rng = np.random.default_rng(7)
    for _ in range(200):
        v = rng.normal(0, 0.05)
        gamma = 10 ** rng.uniform(-2, 2)
        c1 = rng.uniform(0, 2e-3)
        c2 = rng.uniform(0, 1e-2)
        obj = lambda z: 0.5 * (z - v) ** 2 + gamma * (c1 * abs(z) + c2 * abs(z) ** d)
        zs = _golden_min(obj, -abs(v) - 1e-3, abs(v) + 1e-3)
        zp = float(prox_cost(v, gamma, c1, c2, d))
        assert obj(zp) <= obj(zs) + 1e-15
        assert abs(zp - zs) < 1e-7


def test_prox_special_cases():
    v = np.linspace(-0.1, 0.1, 41)
    # c2 = 0: soft thresholding
    np.testing.assert_allclose(prox_cost(v, 2.0, 0.01, 0.0, 1.5),
                               np.sign(v) * np.maximum(np.abs(v) - 0.02, 0), atol=1e-15)
    # d = 2: soft threshold then shrink by 1 / (1 + 2 gamma c2)
    np.testing.assert_allclose(prox_cost(v, 2.0, 0.01, 0.3, 2.0),
                               np.sign(v) * np.maximum(np.abs(v) - 0.02, 0) / (1 + 2 * 2.0 * 0.3),
                               atol=1e-15)
    # dead zone is closed: |v| == gamma c1 maps to 0
    assert prox_cost(0.02, 2.0, 0.01, 0.5, 1.5) == 0.0


def test_projection_is_optimal_against_vertices():
    """p = Proj(v) iff p in B1 and <v - p, u - p> <= 0 for the 2n vertices u = +-e_j
    (the l1 ball is their convex hull)."""
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 37, 200):
        for scale in (0.01, 0.3, 3.0):
            v = rng.normal(0, scale, n)
            p = project_l1(v)
            assert np.abs(p).sum() <= 1 + 1e-12
            if np.abs(v).sum() > 1:
                assert abs(np.abs(p).sum() - 1) < 1e-12
            r = v - p
            # <r, +-e_j - p> = +-r_j - <r, p>
            assert np.max(np.abs(r)) - r @ p <= 1e-12
            th = l1_threshold(v)
            np.testing.assert_allclose(p, np.sign(v) * np.maximum(np.abs(v) - th, 0), atol=1e-15)


def test_projection_brute_force_2d():
    rng = np.random.default_rng(5)
    g = np.linspace(-1, 1, 2001)
    X, Y = np.meshgrid(g, g, indexing="ij")
    inside = np.abs(X) + np.abs(Y) <= 1
    for _ in range(20):
        v = rng.normal(0, 1, 2)
        d2 = (X - v[0]) ** 2 + (Y - v[1]) ** 2
        d2[~inside] = np.inf
        j = np.unravel_index(np.argmin(d2), d2.shape)
        p = project_l1(v)
        assert abs(p[0] - X[j]) <= 2e-3 and abs(p[1] - Y[j]) <= 2e-3


@pytest.mark.parametrize("d", [1.5, 2.0])
def test_conjugate_matches_supremum(d):
    rng = np.random.default_rng(11)
    for _ in range(30):
        c1 = rng.uniform(1e-4, 2e-3)
        c2 = rng.uniform(1e-3, 1e-2)
        y = rng.normal(0, 0.02)
        h = lambda z: -(y * z - c1 * abs(z) - c2 * abs(z) ** d)     # concave objective, negated
        sup = max(-h(_golden_min(h, 0.0, 1e6, 400)), -h(_golden_min(h, -1e6, 0.0, 400)), 0.0)
        assert abs(float(cost_conjugate(y, c1, c2, d)) - sup) <= 1e-9 * max(1.0, abs(sup)) + 1e-12
    assert cost_conjugate(5e-4, 1e-3, 1e-2, 1.5) == 0.0
    assert np.isinf(cost_conjugate(2e-3, 1e-3, 0.0, 1.5))


# ---- joint primal prox: trading cost of Eq. 1 and budget set of Eq. 3 together ----

from oracle.prox import prox_joint, prox_joint_coord  # noqa: E402


@pytest.mark.parametrize("d", [1.3, 1.5, 2.0])
def test_joint_coordinate_matches_direct_minimisation(d):
    """The coordinate problem 0.5 (w - v)^2 + gamma phi(w - a) + mu |w| (two
    kinks, at 0 and at a) against golden-section search of its objective."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        v, a = rng.normal(0, 0.05), rng.normal(0, 0.02)
        gamma, mu = 10 ** rng.uniform(-1, 1), rng.uniform(0, 0.05)
        c1, c2 = rng.uniform(0, 5e-3), rng.uniform(0, 5e-2)
        obj = lambda w: 0.5 * (w - v) ** 2 + gamma * (c1 * abs(w - a) + c2 * abs(w - a) ** d) + mu * abs(w)
        w = float(prox_joint_coord(v, a, mu, gamma, c1, c2, d))
        ws = _golden_min(obj, -abs(v) - abs(a) - 1e-2, abs(v) + abs(a) + 1e-2, iters=300)
        assert obj(w) <= obj(ws) + 1e-15
        assert abs(w - ws) <= 1e-6


def test_joint_prox_reduces_to_projection_and_to_separable_prox():
    """No cost (c1 = c2 = 0): the projection onto the budget set, with mu the
    projection's threshold; a ball that does not bind: a + prox_cost(v - a)."""
    rng = np.random.default_rng(12)
    v = rng.normal(0, 0.1, 40)
    a = rng.normal(0, 0.02, 40)
    w, mu = prox_joint(v, a, 1.0, 0.0, 0.0, 1.5)
    assert np.max(np.abs(w - project_l1(v))) <= 1e-15
    assert abs(mu - l1_threshold(v)) <= 1e-14
    c1, c2 = rng.uniform(0, 2e-3, 40), rng.uniform(0, 2e-2, 40)
    w, mu = prox_joint(v, a, 0.5, c1, c2, 1.5, radius=100.0)
    assert mu == 0.0
    assert np.max(np.abs(w - (a + prox_cost(v - a, 0.5, c1, c2, 1.5)))) <= 1e-15


def test_joint_prox_brute_force_2d():
    """Two assets: the joint prox against a grid search over the ball, and its
    optimality conditions (a subgradient of every term balancing w - v, the
    budget tight when mu > 0)."""
    rng = np.random.default_rng(13)
    d = 1.5
    g = np.linspace(-1.0, 1.0, 2001)
    W1, W2 = np.meshgrid(g, g, indexing="ij")
    inside = np.abs(W1) + np.abs(W2) <= 1.0
    for _ in range(6):
        v = rng.normal(0, 0.8, 2)
        a = rng.normal(0, 0.3, 2)
        gamma, c1, c2 = 0.5, rng.uniform(0.05, 0.3, 2), rng.uniform(0.05, 0.3, 2)
        w, mu = prox_joint(v, a, gamma, c1, c2, d)
        cost = lambda x1, x2: (0.5 * ((x1 - v[0]) ** 2 + (x2 - v[1]) ** 2)
                               + gamma * (c1[0] * np.abs(x1 - a[0]) + c2[0] * np.abs(x1 - a[0]) ** d
                                          + c1[1] * np.abs(x2 - a[1]) + c2[1] * np.abs(x2 - a[1]) ** d))
        grid = np.where(inside, cost(W1, W2), np.inf)
        best = np.unravel_index(np.argmin(grid), grid.shape)
        assert np.abs(w).sum() <= 1.0 + 1e-12
        assert float(cost(w[0], w[1])) <= float(grid[best]) + 1e-12
        assert np.max(np.abs(w - np.array([g[best[0]], g[best[1]]]))) <= 2e-3
        if mu > 0:
            assert abs(np.abs(w).sum() - 1.0) <= 1e-12
