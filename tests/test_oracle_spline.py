"""Pins of the oracle's scatter (Eq. phi_projection with a centred B-spline basis).

Every check is against a fact fixed by mathematics, not against the oracle's own
formula: textbook B-spline values, partition of unity, the box-convolution
recursion, mass conservation, translation covariance and a brute-force support
search.
"""
import json
import os

import numpy as np
import pytest

from oracle import hermes_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_bspline_textbook_values():
    cases = json.load(open(os.path.join(GOLD, "bspline_values.json")))["cases"]
    for c in cases:
        assert O.bspline(c["p"], np.array([c["x"]]))[0] == pytest.approx(c["value"], abs=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_partition_of_unity(p):
    rng = np.random.default_rng(p)
    x = rng.uniform(-3, 3, size=200)
    tot = np.zeros_like(x)
    for l in range(-10, 11):
        tot += O.bspline(p, x - l)
    np.testing.assert_allclose(tot, 1.0, atol=1e-12)


@pytest.mark.parametrize("p", range(2, 8))
def test_box_convolution_recursion(p):
    # M_p = M_{p-1} * M_1 : integrate M_{p-1}(x - y) over y in [-1/2, 1/2)
    rng = np.random.default_rng(10 + p)
    x = rng.uniform(-p / 2.0, p / 2.0, size=25)
    gx, gw = np.polynomial.legendre.leggauss(40)
    # split [-1/2,1/2] at the knots of M_{p-1}(x - y) so each piece is a polynomial
    for xi in x:
        knots = [-0.5, 0.5]
        for k in range(-10, 11):
            y = xi - (k + (0.5 if (p - 1) % 2 == 1 else 0.0))
            if -0.5 < y < 0.5:
                knots.append(y)
        knots = sorted(knots)
        val = 0.0
        for a, b in zip(knots[:-1], knots[1:]):
            yy = 0.5 * (b - a) * gx + 0.5 * (a + b)
            val += 0.5 * (b - a) * np.sum(gw * O.bspline(p - 1, xi - yy))
        assert O.bspline(p, np.array([xi]))[0] == pytest.approx(val, abs=1e-12)


@pytest.mark.parametrize("p", range(1, 9))
def test_node_rule_selects_exact_support(p):
    # brute force: over all nodes of a 1-D periodic grid, those with |u - l| < p/2
    N, L = 32, 100.0
    rng = np.random.default_rng(100 + p)
    pos = rng.uniform(0, L, size=(300, 3)).astype(np.float32)
    first, dist = O.node_rule(pos, N, L, p)
    u = pos.astype(np.float32) * O.scale_f32(N, L)
    for i in range(0, 300, 7):
        for d in range(3):
            ud = float(u[i, d])
            brute = sorted(l % N for l in range(-N, 2 * N) if abs(ud - l) < p / 2.0)
            got = sorted((first[i, d] + o) % N for o in range(p)
                         if O.bspline(p, np.array([dist[i, d, o]]))[0] > 0)
            assert got == brute
            # offsets are u - node exactly
            for o in range(p):
                node = first[i, d] + o
                diff = (ud - node) % N
                diff = diff - N if diff > N / 2 else diff
                assert dist[i, d, o] == pytest.approx(diff, abs=1e-4)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_mass_conservation(p):
    rng = np.random.default_rng(7 + p)
    N, L = 16, 50.0
    pos = rng.uniform(0, L, size=(500, 3)).astype(np.float32)
    w = rng.uniform(0.5, 2.0, size=500)
    eps, sw, sw2 = O.assign(pos, w, N, L, p)
    assert eps.sum() == pytest.approx(w.sum(), rel=1e-12)
    assert sw == pytest.approx(w.sum(), rel=1e-14)
    assert sw2 == pytest.approx((w * w).sum(), rel=1e-14)


def test_translation_by_one_cell_rolls_the_grid():
    # with L = N the scale is exactly 1, so x + 1 is an exact one-cell shift
    N = 16
    L = float(N)
    rng = np.random.default_rng(3)
    # fractions on a 2^-10 lattice keep x + 1 exact in float32 across binades
    pos = (rng.integers(0, N - 2, size=(200, 3))
           + rng.integers(0, 1024, size=(200, 3)) / 1024.0).astype(np.float32)
    e1, _, _ = O.assign(pos, None, N, L, 4)
    e2, _, _ = O.assign((pos + 1.0).astype(np.float32), None, N, L, 4)
    np.testing.assert_array_equal(np.roll(e1, shift=(1, 1, 1), axis=(0, 1, 2)), e2)


def test_point_on_a_node_cubic():
    # a unit point exactly on node (3,5,7) with p=4: weights 1/6, 2/3, 1/6 per axis
    N, L = 16, 16.0
    pos = np.array([[3.0, 5.0, 7.0]], dtype=np.float32)
    eps, _, _ = O.assign(pos, None, N, L, 4)
    w1 = {2: 1 / 6, 3: 2 / 3, 4: 1 / 6}
    for (i, a) in w1.items():
        for (j, b) in {4: 1 / 6, 5: 2 / 3, 6: 1 / 6}.items():
            for (k, c) in {6: 1 / 6, 7: 2 / 3, 8: 1 / 6}.items():
                assert eps[i, j, k] == pytest.approx(a * b * c, abs=1e-15)
    assert np.count_nonzero(eps) == 27


def test_float32_index_rule_is_the_float32_product():
    # the scaled coordinate is the IEEE float32 product, not the float64 one:
    # the largest float32 below L=1000 times fl32(512/1000) rounds to exactly 512,
    # so the point sits on node 512 = 0 (mod N) with t = 0, while a float64
    # product (511.99997) would give node 511 with t close to 1
    N, L = 512, 1000.0
    x = np.nextafter(np.float32(L), np.float32(0))
    first, dist = O.node_rule(np.array([[x, x, x]], dtype=np.float32), N, L, 4)
    assert np.float32(x) * O.scale_f32(N, L) == np.float32(512.0)
    assert first[0, 0] == N - 1                        # nodes 511, 0, 1, 2
    np.testing.assert_array_equal(dist[0, 0], [1.0, 0.0, -1.0, -2.0])
