"""Pins of the oracle's least-squares variant of the Taylor schemes (paper
Sec. 3: the derivatives come from a polynomial fit A x = Q^c through
neighbouring coarse centres, solved in the least-squares sense)."""
import math
from fractions import Fraction as F
from itertools import product

import numpy as np
import pytest
import torch

from oracle import operators as op
from oracle import transfer as tr
from oracle.stencils import multi_indices
from paper_2504_15814_gb300 import workloads as wl

from .test_oracle_operators import _positions, _random_poly, _smooth

LS = op.SCHEME_LS


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("face", [0, 2, 4])
def test_ls_reproduces_polynomials_exactly(order, face):
    rng = np.random.default_rng(500 + 10 * order + face)
    p, k = 6, 3 if face % 2 == 0 else 2
    for sub in (0, 4, 8):
        cpos, fpos = _positions(face, sub, p, k)
        q = _random_poly(rng, order)
        qc, qf = [q(x) for x in cpos], [q(x) for x in fpos]
        outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True, scheme=LS)
        for o, row in zip(outs, rows):
            assert sum(w * qc[c] for c, w in row.items()) == q(fpos[o])
        outs, rows = op.restriction_rows(face, sub, p, k, order, exact=True, scheme=LS)
        for o, row in zip(outs, rows):
            assert sum(w * qf[c] for c, w in row.items()) == q(cpos[o])


def _basis(r, alpha):
    out = F(1)
    for d in range(3):
        out *= F(r[d]) ** alpha[d] / math.factorial(alpha[d])
    return out


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("centre", [(2, 4, 4), (2, 0, 4), (2, 0, 0), (2, 1, 7)])
def test_ls_fit_satisfies_normal_equations(order, centre):
    """For arbitrary data the fitted derivatives x make the residual A x - d
    orthogonal to every column of A (the defining property of least squares),
    checked exactly on random rational data."""
    ext = (6, 9, 9)   # face 0, p = 9, k = 3: (2k, p, p)
    pts = [q for q in op._stencil_support(centre, ext, order) if q != centre]
    rel = tuple(tuple(q[d] - centre[d] for d in range(3)) for q in pts)
    G = op._ls_derivative_weights(rel, order)
    alphas = [a for a in multi_indices(order) if sum(a) > 0]
    rng = np.random.default_rng(sum(centre) + order)
    dvec = [F(int(rng.integers(-50, 51)), int(rng.integers(1, 9))) for _ in pts]
    x = {a: sum(g * dv for g, dv in zip(G[a], dvec)) for a in alphas}
    resid = [sum(_basis(r, a) * x[a] for a in alphas) - dv for r, dv in zip(rel, dvec)]
    for a in alphas:
        assert sum(_basis(r, a) * res for r, res in zip(rel, resid)) == 0
    assert len(pts) > len(alphas)   # over-determined: a genuine fit, not interpolation


def test_ls_equals_fd_where_the_fit_is_square():
    """Taylor-2 restriction fits 2 derivatives through 2 differences on the
    3-point normal window: the least-squares solution is the interpolant, the
    same as the finite-difference reading."""
    for face in (0, 4):
        for sub in (0, 5):
            _, fd = op.restriction_rows(face, sub, 9, 3, 2, exact=True)
            _, ls = op.restriction_rows(face, sub, 9, 3, 2, exact=True, scheme=LS)
            assert fd == ls


def test_ls_differs_from_fd_when_over_determined():
    _, fd = op.interpolation_rows(0, 4, 9, 3, 3, exact=True)
    _, ls = op.interpolation_rows(0, 4, 9, 3, 3, exact=True, scheme=LS)
    assert fd != ls


@pytest.mark.parametrize("order", [2, 3])
def test_ls_rows_sum_to_one_and_inject(order):
    p, k = 9, 3
    for face in (1, 5):
        for sub in (0, 4):
            cpos, fpos = _positions(face, sub, p, k)
            outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True, scheme=LS)
            for o, row in zip(outs, rows):
                assert sum(row.values()) == 1
                if fpos[o] in cpos:
                    assert row == {cpos.index(fpos[o]): 1}


@pytest.mark.parametrize("order,expected", [(2, 3.0), (3, 4.0)])
def test_ls_convergence_order(order, expected):
    items, cl, fl = wl.make_items([1], [-1], [9], [3], [order], 1)
    items["scheme"] = LS
    org = np.array([[0.3, -0.2, 0.1]])
    errs_i, errs_r = [], []
    for H in [0.04 / 2 ** j for j in range(4)]:
        coarse, fine = wl.polynomial_buffers(items, 1, cl, fl, _smooth(H), origins=org / H)
        c, f = coarse.numpy(), fine.numpy()
        out = tr.interpolate(items, 1, c, np.zeros_like(f))
        errs_i.append(np.abs(out[out != 0] - f[out != 0]).max())
        outc = tr.restrict(items, 1, f, np.zeros_like(c))
        errs_r.append(np.abs(outc[outc != 0] - c[outc != 0]).max())
    for errs in (errs_i, errs_r):
        rates = [math.log2(errs[j] / errs[j + 1]) for j in range(len(errs) - 1)]
        assert abs(rates[-1] - expected) < 0.3, rates


def test_ls_equals_dlinear_on_linear_data():
    U = 2
    for order in (2, 3):
        for face in range(6):
            items, cl, fl = wl.make_items([face], [-1], [6], [3], [order], U)
            items["scheme"] = LS
            lin = lambda x: torch.stack([1.5 + 0.3 * x[:, 0] - 0.7 * x[:, 1] + 0.2 * x[:, 2],
                                         -2 + x[:, 0] + x[:, 1] + x[:, 2]], 1)
            coarse, fine = wl.polynomial_buffers(items, U, cl, fl, lin, origins=np.array([[3.0, -2.0, 5.0]]))
            c, f = coarse.numpy(), fine.numpy()
            dl = items.copy()
            dl["order"], dl["scheme"] = 1, 0
            rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
            assert rel(tr.interpolate(items, U, c, f), tr.interpolate(dl, U, c, f)) < 1e-13
            assert rel(tr.restrict(items, U, f, c), tr.restrict(dl, U, f, c)) < 1e-13
