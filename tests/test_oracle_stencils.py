"""Pins of the oracle's 1-D stencil machinery against textbook finite
differences (central, one-sided and staggered Lagrange stencils, e.g. the
standard Fornberg tables) and against the coefficient counts of paper Sec. 3."""
import re
from fractions import Fraction as F
from pathlib import Path

import pytest

from oracle.stencils import (Unsupported, exactness_degree, lagrange_derivative_weights,
                             multi_indices, window)


@pytest.mark.parametrize("points,order,expected", [
    ((-1, 0, 1), 1, (F(-1, 2), 0, F(1, 2))),
    ((-1, 0, 1), 2, (1, -2, 1)),
    ((-2, -1, 0, 1, 2), 1, (F(1, 12), F(-2, 3), 0, F(2, 3), F(-1, 12))),
    ((-2, -1, 0, 1, 2), 2, (F(-1, 12), F(4, 3), F(-5, 2), F(4, 3), F(-1, 12))),
    ((-2, -1, 0, 1, 2), 3, (F(-1, 2), 1, 0, -1, F(1, 2))),
    ((0, 1, 2), 1, (F(-3, 2), 2, F(-1, 2))),
    ((0, 1, 2), 2, (1, -2, 1)),
    ((-2, -1, 0), 1, (F(1, 2), -2, F(3, 2))),
    ((0, 1, 2, 3, 4), 1, (F(-25, 12), 4, -3, F(4, 3), F(-1, 4))),
    ((0, 1, 2, 3, 4), 2, (F(35, 12), F(-26, 3), F(19, 2), F(-14, 3), F(11, 12))),
    ((0, 1, 2, 3, 4), 3, (F(-5, 2), 9, -12, 7, F(-3, 2))),
    ((-1, 0, 1, 2), 1, (F(-1, 3), F(-1, 2), 1, F(-1, 6))),
    ((-1, 0, 1, 2), 2, (1, -2, 1, 0)),
    ((-1, 0, 1, 2), 3, (-1, 3, -3, 1)),
])
def test_textbook_weights(points, order, expected):
    assert lagrange_derivative_weights(points, 0, order) == tuple(F(e) for e in expected)


def test_weights_annihilate_lower_and_reproduce_power():
    # sum_i w_i x_i^r = r! delta_{r,order} for r < len(points): the defining moments
    pts = (-3, -1, 0, 2, 5)
    for order in range(1, 4):
        w = lagrange_derivative_weights(pts, 0, order)
        for r in range(len(pts)):
            mom = sum(wi * F(x) ** r for wi, x in zip(w, pts))
            assert mom == (F(6) if r == order == 3 else F(2) if r == order == 2 else F(1) if r == order else 0)


@pytest.mark.parametrize("centre,lo,hi,E,expected", [
    (4, 0, 8, 3, range(2, 7)),      # centred 5-point
    (0, 0, 8, 3, range(0, 5)),      # shifted inward at the low end
    (1, 0, 8, 3, range(0, 5)),
    (8, 0, 8, 3, range(4, 9)),      # shifted inward at the high end
    (4, 0, 8, 2, range(3, 6)),      # centred 3-point
    (0, 0, 8, 1, range(0, 3)),      # first derivative for mixed terms still uses 3 points
    (1, 0, 3, 3, range(0, 4)),      # range of 4 < 5 but >= E+1: whole range
    (-1, -3, 2, 3, range(-3, 2)),   # normal window about the coarse layer next to the interface, k = 3
    (-1, -2, 1, 3, range(-2, 2)),   # same for k = 2: whole range of 4
])
def test_window_rule(centre, lo, hi, E, expected):
    assert window(centre, lo, hi, E) == tuple(expected)


def test_window_unsupported():
    with pytest.raises(Unsupported):
        window(0, -1, 0, 2)   # k = 1 normal range cannot hold 3 points


def _golden():
    out = {}
    for line in (Path(__file__).parent / "golden" / "paper_facts.txt").read_text().splitlines():
        m = re.match(r"(\w+)\s*=\s*([^#]+)", line)
        if m:
            out[m.group(1)] = m.group(2).strip()
    return out


def test_coefficient_counts_match_paper():
    gold = _golden()
    assert len(multi_indices(2)) == int(gold["taylor_coefficients_order2"])
    assert len(multi_indices(3)) == int(gold["taylor_coefficients_order3"])


def test_exactness_degree():
    # pure derivatives must be exact up to the scheme order; the mixed u_xy of
    # Taylor-3 only up to degree 2 along each axis, u_xyz up to degree 1
    assert exactness_degree((1, 0, 0), 0, 3) == 3
    assert exactness_degree((1, 1, 0), 0, 3) == 2
    assert exactness_degree((1, 1, 1), 2, 3) == 1
    assert exactness_degree((2, 1, 0), 1, 3) == 1
