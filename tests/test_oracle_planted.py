"""The oracle's pins catch plausible mistakes.  Each test plants one mistake
in the oracle (on the CPU, by monkeypatching) and checks that a pin that does
not reuse the oracle's formulas fails: exact reproduction of polynomials at
generator-placed centres, or the textbook stencil weights."""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import operators as op
from oracle import stencils as st
from paper_2504_15814_gb300 import workloads as wl


def _positions(face, sub, p, k):
    items, _, _ = wl.make_items([face], [sub], [p], [k], [2], 1)
    cpos, _, fpos, _ = wl.volume_positions(items, 1, np.zeros((1, 3)))
    snap = lambda a: [tuple(F(float(v)).limit_denominator(6) for v in row) for row in a.numpy()]
    return snap(cpos), snap(fpos)


def _reproduces(order, face=0, sub=4, p=6, k=3, seed=0):
    """True iff interpolation and restriction reproduce a random polynomial of
    the scheme's degree exactly (the pin of test_oracle_operators)."""
    rng = np.random.default_rng(seed)
    terms = {(a, b, c): F(int(rng.integers(-9, 10)), int(rng.integers(1, 7)))
             for a in range(order + 1) for b in range(order + 1 - a) for c in range(order + 1 - a - b)}
    q = lambda x: sum(cf * x[0] ** a * x[1] ** b * x[2] ** c for (a, b, c), cf in terms.items())
    cpos, fpos = _positions(face, sub, p, k)
    qc, qf = [q(x) for x in cpos], [q(x) for x in fpos]
    outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True)
    ok = all(sum(w * qc[c] for c, w in row.items()) == q(fpos[o]) for o, row in zip(outs, rows))
    outs, rows = op.restriction_rows(face, sub, p, k, order, exact=True)
    ok &= all(sum(w * qf[c] for c, w in row.items()) == q(cpos[o]) for o, row in zip(outs, rows))
    return ok


@pytest.mark.parametrize("order", [2, 3])
def test_unplanted_oracle_passes(order):
    assert _reproduces(order)


@pytest.mark.parametrize("order", [2, 3])
def test_dropped_mixed_terms_are_caught(order, monkeypatch):
    real = st.multi_indices
    monkeypatch.setattr(op, "multi_indices", lambda m: [a for a in real(m) if sum(1 for v in a if v) <= 1])
    assert not _reproduces(order)


@pytest.mark.parametrize("order", [2, 3])
def test_wrong_taylor_factorial_is_caught(order, monkeypatch):
    monkeypatch.setattr(op, "_factorial", lambda n: 1)
    assert not _reproduces(order)


@pytest.mark.parametrize("order", [2, 3])
def test_flipped_offset_sign_is_caught(order, monkeypatch):
    real = op.taylor_row
    monkeypatch.setattr(op, "taylor_row", lambda c, ext, off, m, num: real(c, ext, [-o for o in off], m, num))
    assert not _reproduces(order)


def test_window_too_short_is_caught(monkeypatch):
    # exactness degree one too low: 3-point windows where Taylor-3 needs 5
    # (for Taylor-2 the odd-length rule keeps 3 points, so the same slip is
    # harmless there)
    real = op.exactness_degree
    monkeypatch.setattr(op, "exactness_degree", lambda alpha, d, m: max(real(alpha, d, m) - 1, 1))
    assert not _reproduces(3)


def test_transposed_axes_are_caught(monkeypatch):
    # Taylor offsets applied to the wrong axes (t0 and t1 swapped)
    real_row = op.taylor_row

    def row(c, ext, off, m, num):
        off2 = list(off)
        off2[1], off2[2] = off2[2], off2[1]
        return real_row(c, ext, off2, m, num)
    monkeypatch.setattr(op, "taylor_row", row)
    assert not _reproduces(3, face=1, sub=5)


@pytest.mark.parametrize("order", [2, 3])
def test_wrong_lagrange_weights_are_caught(order, monkeypatch):
    # first-derivative weights evaluated one centre off the expansion point
    real = st.lagrange_derivative_weights.__wrapped__

    def shifted(points, x0, r):
        return real(points, x0 + 1 if r == 1 else x0, r)
    monkeypatch.setattr(op, "lagrange_derivative_weights", shifted)
    assert not _reproduces(order)
