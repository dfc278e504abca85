"""Pins of the oracle's single-output evaluators.

``transfer.interpolate_one`` (one fine ghost element of P Q^c, Sec. 2) is the
checker of the full-size sampled GPU tests, so it is held to the whole-buffer
``transfer.interpolate`` -- itself pinned by exact reproduction of polynomials
and the d-linear identities -- over every ghost element of a small mixed
batch: all six faces, whole-face and single-subface items (Sec. 2: one call
per 1/9 block), overlaps 1..3, patch sizes that are and are not multiples of
3, all orders and both derivative schemes.  A planted index mistake (a
transposed tangential axis, a wrong subface array) must fail it.
"""
import numpy as np
import pytest

from oracle import transfer as tr
from paper_2504_15814_gb300 import workloads as wl


def _mixed_batch(U, seed):
    faces = [0, 1, 2, 3, 4, 5, 0, 3, 1, 5, 2, 4]
    subs = [-1, 4, 0, 8, -1, 2, 6, -1, 3, 5, 7, 1]
    ps = [6, 9, 4, 7, 5, 9, 6, 8, 9, 6, 12, 5]
    ks = [3, 2, 2, 3, 2, 3, 1, 2, 3, 2, 3, 3]
    orders = [3, 2, 3, 1, 2, 3, 1, 3, 2, 3, 3, 1]
    items, cl, fl = wl.make_items(faces, subs, ps, ks, orders, U)
    # least-squares derivatives on a few Taylor items (scheme 1, Sec. 3)
    for i in (1, 5, 9):
        items[i]["scheme"] = 1
    rng = np.random.default_rng(seed)
    return items, rng.standard_normal(cl), rng.standard_normal(fl)


def _owner(items, U, e):
    for it in items:
        p, k = int(it["patch_size"]), int(it["overlap"])
        n = 2 * k * p * p * U * (9 if int(it["subface"]) < 0 else 1)
        fo = int(it["fine_offset"])
        if fo <= e < fo + n:
            return it
    raise AssertionError(e)


def test_interpolate_one_matches_interpolate_everywhere():
    U = 2
    items, coarse, fine = _mixed_batch(U, 7)
    marker = np.full_like(fine, np.nan)
    out = tr.interpolate(items, U, coarse, marker)
    written = np.flatnonzero(~np.isnan(out))
    expected = sum(int(it["overlap"]) * int(it["patch_size"]) ** 2 * U * (9 if int(it["subface"]) < 0 else 1)
                   for it in items)
    assert written.size == expected
    scale = np.abs(out[written]).max()
    for e in written:
        got = tr.interpolate_one(_owner(items, U, int(e)), U, coarse, int(e))
        assert abs(got - out[e]) <= 1e-14 * scale, (int(e), got, out[e])


def test_interpolate_one_catches_a_wrong_subface_array():
    """The same element evaluated as if it belonged to the neighbouring
    subface's array differs (the check is sensitive to the block index)."""
    U = 1
    items, cl, fl = wl.make_items([2], [-1], [6], [3], [3], U)
    rng = np.random.default_rng(3)
    coarse = rng.standard_normal(cl)
    out = tr.interpolate(items, U, coarse, np.full(fl, np.nan))
    n = 2 * 3 * 36 * U
    e = int(np.flatnonzero(~np.isnan(out[:n]))[5])
    assert abs(tr.interpolate_one(items[0], U, coarse, e) - out[e]) < 1e-14
    assert abs(tr.interpolate_one(items[0], U, coarse, e + n) - out[e]) > 1e-6


@pytest.mark.parametrize("seed", [1, 2])
def test_restrict_one_matches_restrict_everywhere(seed):
    U = 2
    items, coarse, fine = _mixed_batch(U, seed)
    out = tr.restrict(items, U, fine, np.full_like(coarse, np.nan))
    written = np.flatnonzero(~np.isnan(out))
    scale = np.abs(out[written]).max()
    starts = [int(it["coarse_offset"]) for it in items]
    for e in written:
        it = items[int(np.searchsorted(starts, e, side="right")) - 1]
        assert abs(tr.restrict_one(it, U, fine, int(e)) - out[e]) <= 1e-14 * scale
