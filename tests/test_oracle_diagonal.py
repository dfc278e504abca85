"""Pins of the diagonal (edge and vertex) halo reading of the oracle.

The paper's code has no diagonal halo data (Sec. 2); the reading here widens
each subface's ghost half by k volumes on each tangential side and fills the
widened strip from the same coarse face array by the same rule (nearest
coarse centre, its stencils, Taylor's formula; d-linear tensor product with
extrapolation past the face edge).  Pinned by: exact reproduction of
polynomials of the scheme's degree at every widened volume (Taylor's formula
with exact derivatives holds at any offset, Sec. 3); linear exactness of
d-linear; equality with the ordinary rows of the neighbouring subface where
the strip lies over it (same physical position); the strip's size."""
import random
from fractions import Fraction

import pytest

from oracle import geometry as g
from oracle import operators as op


def _poly(rng, degree):
    terms = []
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                terms.append((a, b, c, Fraction(rng.randint(-9, 9), rng.randint(1, 5))))
    return lambda x: sum(w * x[0] ** a * x[1] ** b * x[2] ** c for a, b, c, w in terms)


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("face,sub,p,k", [(0, 4, 6, 3), (1, 0, 6, 2), (5, 8, 9, 3), (2, 2, 7, 3)])
def test_diagonal_rows_reproduce_polynomials(face, sub, p, k, order):
    rng = random.Random(100 * face + 10 * sub + order)
    q = _poly(rng, order)
    ext = g.extents(face, p, k)
    cpos = {g.flat(ext, idx): g.coarse_centre(face, p, k, idx) for idx in g.all_indices(ext)}
    outs, rows = op.diagonal_interpolation_rows(face, sub, p, k, order, exact=True)
    assert len(outs) == k * ((p + 2 * k) ** 2 - p * p)
    for idx, row in zip(outs, rows):
        xf = g.fine_centre(face, p, k, sub, idx)
        assert sum(w * q(cpos[c]) for c, w in row.items()) == q(xf)


def test_degree_above_the_order_is_not_reproduced():
    face, sub, p, k, order = 0, 0, 6, 3, 2
    ext = g.extents(face, p, k)
    cpos = {g.flat(ext, idx): g.coarse_centre(face, p, k, idx) for idx in g.all_indices(ext)}
    cube = lambda x: x[1] ** 3
    outs, rows = op.diagonal_interpolation_rows(face, sub, p, k, order, exact=True)
    misses = sum(sum(w * cube(cpos[c]) for c, w in row.items()) != cube(g.fine_centre(face, p, k, sub, idx))
                 for idx, row in zip(outs, rows))
    assert misses > 0


@pytest.mark.parametrize("order", [1, 2, 3])
def test_strip_over_a_neighbour_equals_its_ghost_rows(order):
    """Subface 4's strip at t0 indices p..p+k-1 lies over subface 5's ghost
    volumes 0..k-1 (same physical centres): identical rows."""
    face, p, k = 2, 6, 3
    n, t0, t1 = g.axes(face)
    outs, rows = op.diagonal_interpolation_rows(face, 4, p, k, order, exact=True)
    ref_outs, ref_rows = op.interpolation_rows(face, 5, p, k, order, exact=True)
    ext = g.extents(face, p, k)
    ref = dict(zip(ref_outs, ref_rows))
    checked = 0
    for idx, row in zip(outs, rows):
        if p <= idx[t0] < p + k and 0 <= idx[t1] < p:
            j = list(idx)
            j[t0] = idx[t0] - p
            assert {c: w for c, w in row.items() if w} == {c: w for c, w in ref[g.flat(ext, tuple(j))].items() if w}
            checked += 1
    assert checked == k * k * p
