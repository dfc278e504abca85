"""Pins of the oracle for patch sizes that are not multiples of 3 (the paper
notes its methods do slightly better when p is one, Sec. 5.3, so other sizes
are allowed).  A coarse volume a covers fine global indices 3a .. 3a+2 and its
centre coincides with fine 3a + 1; a subface boundary can cut a coarse volume,
which then belongs to the subface holding 3a + 1.

Checked against facts that do not reuse the oracle's formulas: exact
reproduction of polynomials of the scheme's degree at centres placed by the
workload generator, the ownership partition (every fine-side coarse volume
restricted exactly once, at a coincident fine centre), a hand-derived d-linear
row on a cut volume, and the convergence order on a smooth field.  Also
pinned here: overlaps k > 3 (deeper ghost layers), which the oracle's
geometry covers although the GPU path stops at k = 3."""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import geometry as g
from oracle import operators as op
from oracle import transfer as tr
from paper_2504_15814_gb300 import workloads as wl

from .test_oracle_operators import _positions, _random_poly, _smooth

PS = (4, 5, 7, 8)


@pytest.mark.parametrize("scheme", [op.SCHEME_FD, op.SCHEME_LS])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("p", PS)
def test_taylor_reproduces_polynomials(p, order, scheme):
    rng = np.random.default_rng(1000 * p + 10 * order + scheme)
    k = 3 if p % 2 else 2
    face = (p + order) % 6
    for sub in (0, 2, 4, 6, 7):
        cpos, fpos = _positions(face, sub, p, k)
        q = _random_poly(rng, order)
        qc = [q(x) for x in cpos]
        qf = [q(x) for x in fpos]
        outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True, scheme=scheme)
        assert len(outs) == k * p * p
        for o, row in zip(outs, rows):
            assert sum(w * qc[c] for c, w in row.items()) == q(fpos[o])
        outs, rows = op.restriction_rows(face, sub, p, k, order, exact=True, scheme=scheme)
        for o, row in zip(outs, rows):
            assert sum(w * qf[c] for c, w in row.items()) == q(cpos[o])


@pytest.mark.parametrize("p", PS)
def test_dlinear_exact_on_linear(p):
    rng = np.random.default_rng(77 + p)
    for face, k in ((1, 1), (3, 2), (5, 3)):
        for sub in range(9):
            cpos, fpos = _positions(face, sub, p, k)
            q = _random_poly(rng, 1)
            outs, rows = op.interpolation_rows(face, sub, p, k, 1, exact=True)
            for o, row in zip(outs, rows):
                assert sum(w * q(cpos[c]) for c, w in row.items()) == q(fpos[o])
            outs, rows = op.restriction_rows(face, sub, p, k, 1, exact=True)
            for o, row in zip(outs, rows):
                assert sum(w * q(fpos[c]) for c, w in row.items()) == q(cpos[o])


@pytest.mark.parametrize("p", PS + (6, 9))
def test_ownership_partitions_the_halo(p):
    """The nine subfaces restrict disjoint sets of coarse volumes that cover
    the fine-side half of the coarse array, each at a fine centre of its
    own subface that coincides with it tangentially."""
    k = 2
    for face in (0, 4):
        n, t0, t1 = g.axes(face)
        side = g.coarse_side(face)
        ext = g.extents(face, p, k)
        halo = [idx for idx in g.all_indices(ext) if (idx[n] - k + F(1, 2)) * side < 0]
        seen = []
        for sub in range(9):
            cpos, fpos = _positions(face, sub, p, k)
            fine_t = {(x[t0], x[t1]) for x in fpos}
            mine = g.coarse_halo_indices(face, p, k, sub)
            for idx in mine:
                xc = cpos[g.flat(ext, idx)]
                assert (xc[t0], xc[t1]) in fine_t
            seen += mine
        assert sorted(seen) == sorted(halo)
        if p % 3 == 0:
            assert all(len(g.coarse_halo_indices(face, p, k, s)) == k * (p // 3) ** 2 for s in range(9))


def test_hand_derived_dlinear_row_on_a_cut_volume():
    """p = 4, face 0 (normal x, t0 = y, t1 = z), k = 2, subface 4 (s0 = s1 = 1)
    holds fine global tangential indices 4 .. 7.  Coarse volume a = 1 covers
    fine 3, 4, 5 and its centre coincides with fine 4 (local 0): subface 4
    owns it but holds only fine 4 and 5 of it, and the least-squares line
    through two points evaluated at one of them is that point, so along y and
    z the row injects local 0.  Along x (coarse on the low side; fine own
    layers at +1/6, +1/2 in units of H, coarse halo layer 0 at +1/2) the line
    through the own layers takes layer 3 (x = +1/2) alone.  Coarse volume
    a = 2 covers fine 6, 7, 8 (centre at fine 7, local 3): owner (3*2+1)//4 = 1,
    and only fine 6 and 7 lie in the subface: injection of local 3."""
    p, k, face, sub = 4, 2, 0, 4
    ext = g.extents(face, p, k)
    outs, rows = op.restriction_rows(face, sub, p, k, 1, exact=True)
    rows = dict(zip(outs, rows))
    # coarse halo layer 0 on the fine side is normal index k = 2; fine layer k + 1 = 3 sits at +1/2
    for (ay, az), (qy, qz) in (((1, 1), (0, 0)), ((2, 1), (3, 0)), ((1, 2), (0, 3)), ((2, 2), (3, 3))):
        row = {c: w for c, w in rows[g.flat(ext, (2, ay, az))].items() if w != 0}
        assert row == {g.flat(ext, (3, qy, qz)): 1}
    assert len(outs) == k * 2 * 2


@pytest.mark.parametrize("p", (5, 7))
def test_restrict_one_matches_restrict(p):
    U = 2
    items, cl, fl = wl.make_items([2, 3], [-1, -1], [p, p], [3, 2], [3, 1], U)
    rng = np.random.default_rng(p)
    fine = rng.standard_normal(fl)
    out = tr.restrict(items, U, fine, np.zeros(cl))
    written = np.flatnonzero(out)
    assert written.size == sum(p * p * int(it["overlap"]) * U for it in items)
    for e in rng.choice(written, 40, replace=False):
        it = items[0] if e < int(items[1]["coarse_offset"]) else items[1]
        assert abs(tr.restrict_one(it, U, fine, int(e)) - out[e]) < 1e-13 * np.abs(out).max()


@pytest.mark.parametrize("order,expected", [(1, 2.0), (2, 3.0), (3, 4.0)])
def test_convergence_order_p8(order, expected):
    """The measured max-norm rate on a whole hanging face with p = 8 matches
    the scheme's order, as for multiples of 3 (Sec. 5.1)."""
    items, cl, fl = wl.make_items([2], [-1], [8], [3], [order], 1)
    org = np.array([[0.3, -0.2, 0.1]])
    errs_i, errs_r = [], []
    for H in [0.04 / 2 ** j for j in range(4)]:
        coarse, fine = wl.polynomial_buffers(items, 1, cl, fl, _smooth(H), origins=org / H)
        c, f = coarse.numpy(), fine.numpy()
        out = tr.interpolate(items, 1, c, np.zeros_like(f))
        ghost = out != 0
        errs_i.append(np.abs(out[ghost] - f[ghost]).max())
        outc = tr.restrict(items, 1, f, np.zeros_like(c))
        halo = outc != 0
        errs_r.append(np.abs(outc[halo] - c[halo]).max())
    for errs in (errs_i, errs_r):
        rates = [math.log2(errs[j] / errs[j + 1]) for j in range(len(errs) - 1)]
        assert abs(rates[-1] - expected) < 0.3, rates


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("k", [4, 5])
def test_deeper_overlaps_reproduce_polynomials(k, order):
    """Overlaps beyond the paper's 3 (fine ghost layers then have nearest
    coarse centres in deeper coarse layers; restriction injects every coarse
    layer whose centre coincides with a fine one): exact on polynomials of
    the scheme's degree (linear for d-linear)."""
    rng = np.random.default_rng(50 * k + order)
    p = 9
    for face, sub in ((0, 4), (4, 0), (2, 8)):
        cpos, fpos = _positions(face, sub, p, k)
        q = _random_poly(rng, order)
        outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True)
        assert len(outs) == k * p * p
        for o, row in zip(outs, rows):
            assert sum(w * q(cpos[c]) for c, w in row.items()) == q(fpos[o])
        outs, rows = op.restriction_rows(face, sub, p, k, order, exact=True)
        assert len(outs) == k * (p // 3) ** 2
        for o, row in zip(outs, rows):
            assert sum(w * q(fpos[c]) for c, w in row.items()) == q(cpos[o])
