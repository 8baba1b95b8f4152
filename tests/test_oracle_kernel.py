"""Pins of the oracle's kernel, lattice sums and Morton code (Eqs. 9, 16, 17).

These fix the oracle against closed forms and the mathematics, never
against itself: quadrature of the kernel, finite differences of its
derivative, the continuum limits of the lattice sums and the bit layout
printed in Eq. 9."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("h", [0.065, 1.0, 3.7])
def test_kernel_integrates_to_one(h):
    # Eq. 16 with alpha_3 = 21 / (16 pi h^3): the 3-D integral over the
    # support 2h is one (partition of unity).
    val, err = integrate.quad(lambda r: 4.0 * math.pi * r * r * O.W(r, h), 0.0, 2.0 * h,
                              epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-10


def test_printed_normalisation_is_not_a_unit_integral():
    # Eq. 17 prints 21 / (6 pi h^3); against the reading above it differs by
    # the factor 16 / 6, so the printed value integrates to 8/3.
    h = 1.0
    assert O.alpha3(h) * (16.0 / 6.0) == pytest.approx(21.0 / (6.0 * math.pi), rel=1e-15)


def test_kernel_special_values():
    h = 0.5
    a = 21.0 / (16.0 * math.pi * h ** 3)
    assert O.W(0.0, h) == pytest.approx(a, rel=1e-15)
    assert O.W(h, h) == pytest.approx(a * 3.0 / 16.0, rel=1e-14)      # (1/2)^4 * 3
    assert O.W(2.0 * h, h) == 0.0
    assert O.W(2.5 * h, h) == 0.0
    assert O.dW(0.0, h) == 0.0
    assert O.dW(2.0 * h, h) == 0.0
    # dW/dr is extremal at q = 1/2 ... derivative of q(1-q/2)^3 vanishes at q = 1/2
    q = np.linspace(0.01, 1.99, 397)
    vals = np.array([O.dW(x * h, h) for x in q])
    assert q[np.argmin(vals)] == pytest.approx(0.5, abs=0.006)


@pytest.mark.parametrize("h", [0.065, 1.0])
def test_kernel_derivative_matches_finite_differences(h):
    for q in np.linspace(0.05, 1.95, 39):
        r = q * h
        eps = 1e-6 * h
        fd = (O.W(r + eps, h) - O.W(r - eps, h)) / (2 * eps)
        assert O.dW(r, h) == pytest.approx(fd, rel=1e-7, abs=1e-9 * O.alpha3(h) / h)


def test_lattice_sums_reach_their_continuum_limits():
    # Cubic lattice: sum W dx^3 -> integral of W = 1.
    # Square lattice (3-D kernel): sum W dx^2 -> 2 pi int W r dr = 3 / (4 h).
    # Line lattice: sum W dx -> int W dr = 7 / (4 pi h^2).
    dx, h = 1.0, 4.0
    assert O.lattice_sum(dx, h, 3) * dx ** 3 == pytest.approx(1.0, abs=2e-5)
    assert O.lattice_sum(dx, h, 2) * dx ** 2 == pytest.approx(0.75 / h, rel=1e-4)
    assert O.lattice_sum(dx, h, 1) * dx == pytest.approx(7.0 / (4.0 * math.pi * h * h), rel=2e-4)
    # and the error shrinks as h / dx grows
    for dim, lim in ((3, lambda k: 1.0), (2, lambda k: 0.75 / k), (1, lambda k: 7.0 / (4.0 * math.pi * k * k))):
        e = [abs(O.lattice_sum(1.0, k, dim) / lim(k) - 1.0) for k in (2.0, 3.0, 4.0, 6.0)]
        assert e[0] > e[1] > e[2] > e[3]


def test_morton_code_matches_eq9_bit_layout():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_eq9.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) >= 8
    for x, y, z, code in rows:
        assert O.morton3(int(x), int(y), int(z)) == int(code)
