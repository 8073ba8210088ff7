"""Pins of the oracle's cut-off function K (Eq. 12-15) and transition
function W (Eq. 16-17) against facts the paper and the mathematics fix,
not against the oracle's own formula."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle

GAMMA = 0.1


def test_K_boundary_values():
    # Eq. 12: 0 below x = 0, 1 from x = 1 on; continuous at both ends
    assert oracle.K(-1e-3) == 0.0
    assert oracle.K(0.0) == 0.0
    assert oracle.K(1.0) == 1.0
    assert oracle.K(5.0) == 1.0
    assert abs(oracle.K(1.0 - 1e-9) - 1.0) < 1e-12
    assert abs(oracle.K(1e-9)) < 1e-30


def test_K_half_and_symmetry():
    # the polynomial of Eq. 12 is antisymmetric about (1/2, 1/2):
    # K(x) + K(1 - x) = 1, hence K(1/2) = 1/2
    assert abs(oracle.K(0.5) - 0.5) < 1e-15
    x = np.linspace(0.0, 1.0, 101)
    assert np.max(np.abs(oracle.K(x) + oracle.K(1.0 - x) - 1.0)) < 1e-13


def test_K_derivatives_vanish_to_third_order():
    # Sect. 2.1: derivatives up to third order are zero at x = 0 and x = 1, so
    # K(d) ~ c d^4 and 1 - K(1 - d) ~ c d^4 with c = 35
    for d in (1e-2, 1e-3):
        assert abs(oracle.K(d) / d**4 - 35.0) < 300 * d
        assert abs((1.0 - oracle.K(1.0 - d)) / d**4 - 35.0) < 300 * d
    # first derivative via central differences is 0 at both ends too (up to
    # the rounding of the degree-7 polynomial near x = 1, ~1e-14 / h)
    h = 1e-6
    for x0 in (0.0, 1.0):
        dk = (oracle.K(x0 + h) - oracle.K(x0 - h)) / (2 * h)
        assert abs(dk) < 1e-7


def test_K_integral_and_monotone():
    val, _ = quad(lambda t: float(oracle.K(t)), 0.0, 1.0)
    assert abs(val - 0.5) < 1e-12
    x = np.linspace(0.0, 1.0, 2001)
    assert np.all(np.diff(oracle.K(x)) >= 0.0)


def test_dKdx_matches_difference_quotient():
    h = 1e-6
    for x in (0.1, 0.3, 0.5, 0.77, 0.95):
        fd = (oracle.K(x + h) - oracle.K(x - h)) / (2 * h)
        assert abs(oracle.dKdx(x) - fd) < 1e-8


def test_K_of_s_maps_radii():
    # Eq. 13-15: K = 0 at s = r_in, 1/2 halfway, 1 at s = r_cut
    r_cut = 0.01
    r_in = GAMMA * r_cut
    assert oracle.K_of_s(r_in, r_cut, GAMMA) == 0.0
    assert abs(oracle.K_of_s(0.5 * (r_in + r_cut), r_cut, GAMMA) - 0.5) < 1e-14
    assert oracle.K_of_s(r_cut, r_cut, GAMMA) == 1.0


def _W_by_quadrature(y, g):
    """W solves K = W - y dW/dy (Eq. 9) with W = 1 for y >= 1, i.e.
    W(y) = y (1 + int_y^1 K(t)/t^2 dt) -- an independent route to W."""
    if y >= 1.0:
        return 1.0
    Ky = lambda t: float(oracle.K((t - g) / (1.0 - g)))
    lo = max(y, g)
    val, _ = quad(lambda t: Ky(t) / (t * t), lo, 1.0, limit=200,
                  epsabs=1e-14, epsrel=1e-13)
    return y * (1.0 + val)


@pytest.mark.parametrize("y", [0.03, 0.1, 0.2, 0.37, 0.5, 0.55, 0.8, 0.99, 1.3])
def test_W_closed_form_matches_eq9(y):
    # the closed form of Eq. 16-17 (numerator sign of G reversed) must agree
    # with the integral of Eq. 9; with the printed sign it is off by O(1)
    assert abs(oracle.W(y, GAMMA) - _W_by_quadrature(y, GAMMA)) < 1e-10


def test_W_pinned_values():
    # W(0.5; 0.1) and the slope below r_in, both by quadrature of Eq. 9
    assert abs(oracle.W(0.5, GAMMA) - 0.871550559274) < 1e-11
    c = oracle.W_inner_slope(GAMMA)
    assert abs(c - 1.98763380440) < 1e-10
    assert abs(c - _W_by_quadrature(GAMMA * 0.5, GAMMA) / (GAMMA * 0.5)) < 1e-9
    # gamma -> 0: slope -> 7/3 (the y < gamma branch of Eq. 16)
    assert abs(oracle.W_inner_slope(1e-4) - 7.0 / 3.0) < 1e-2


def test_W_continuous_and_K_relation():
    g = GAMMA
    for y0 in (g, 1.0):
        assert abs(oracle.W(y0 - 1e-12, g) - oracle.W(y0 + 1e-12, g)) < 1e-9
    # K = W - y W' (Eq. 9) by central differences inside (gamma, 1)
    h = 1e-6
    for y in (0.15, 0.3, 0.55, 0.7, 0.9):
        Wp = (oracle.W(y + h, g) - oracle.W(y - h, g)) / (2 * h)
        K = oracle.K((y - g) / (1 - g))
        assert abs(oracle.W(y, g) - y * Wp - K) < 1e-7
