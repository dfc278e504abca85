"""Pins of the oracle's operators (paper Secs. 2, 3, 5.1 and the appendix
"Testing") against closed forms and invariants that do not reuse the oracle's
own formulas: exact reproduction of polynomials of the scheme's degree at
cell centres placed by the (independently written) workload generator,
constants preserved, injection at coincident centres, hand-derived weights,
the d-linear tensor product = assembled matrix identity, Taylor = d-linear on
linear data, mirror and rotation equivariance, the matrix sizes printed in
Sec. 2, and the measured convergence order on a smooth field."""
import math
from fractions import Fraction as F

import numpy as np
import pytest
import torch

from oracle import geometry as g
from oracle import operators as op
from oracle import transfer as tr
from paper_2504_15814_gb300 import workloads as wl


def _positions(face, sub, p, k):
    """(coarse centres, fine centres of subface sub) from the workload generator,
    snapped to exact multiples of H/6."""
    items, _, _ = wl.make_items([face], [sub], [p], [k], [2], 1)
    cpos, _, fpos, _ = wl.volume_positions(items, 1, np.zeros((1, 3)))
    snap = lambda a: [tuple(F(float(v)).limit_denominator(6) for v in row) for row in a.numpy()]
    return snap(cpos), snap(fpos)


def _random_poly(rng, degree):
    terms = {}
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                terms[(a, b, c)] = F(int(rng.integers(-9, 10)), int(rng.integers(1, 7)))
    return lambda x: sum(cf * x[0] ** a * x[1] ** b * x[2] ** c for (a, b, c), cf in terms.items())


SUBS_SAMPLE = (0, 1, 4, 5, 8)


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("face", range(6))
def test_interpolation_reproduces_polynomials_exactly(order, face):
    rng = np.random.default_rng(100 * order + face)
    p, k = 6, 2 if face % 2 else 3
    for sub in SUBS_SAMPLE:
        cpos, fpos = _positions(face, sub, p, k)
        q = _random_poly(rng, order)
        qc = [q(x) for x in cpos]
        outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True)
        assert len(outs) == k * p * p
        for o, row in zip(outs, rows):
            assert sum(w * qc[c] for c, w in row.items()) == q(fpos[o])


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("face", range(6))
def test_restriction_reproduces_polynomials_exactly(order, face):
    rng = np.random.default_rng(200 * order + face)
    p, k = 6, 3 if face % 2 else 2
    for sub in SUBS_SAMPLE:
        cpos, fpos = _positions(face, sub, p, k)
        q = _random_poly(rng, order)
        qf = [q(x) for x in fpos]
        outs, rows = op.restriction_rows(face, sub, p, k, order, exact=True)
        assert len(outs) == k * (p // 3) ** 2
        for o, row in zip(outs, rows):
            assert sum(w * qf[c] for c, w in row.items()) == q(cpos[o])


@pytest.mark.parametrize("order", [2, 3])
def test_order_is_not_higher_than_claimed(order):
    # a monomial of degree m+1 along the normal is not reproduced everywhere
    face, sub, p, k = 0, 4, 6, 3
    cpos, fpos = _positions(face, sub, p, k)
    q = lambda x: x[0] ** (order + 1)
    outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True)
    errs = [sum(w * q(cpos[c]) for c, w in row.items()) - q(fpos[o]) for o, row in zip(outs, rows)]
    assert any(e != 0 for e in errs)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("face", range(6))
def test_dlinear_exact_on_linear(face, k):
    rng = np.random.default_rng(300 + 10 * face + k)
    p = 6
    for sub in range(9):
        cpos, fpos = _positions(face, sub, p, k)
        q = _random_poly(rng, 1)
        outs, rows = op.interpolation_rows(face, sub, p, k, 1, exact=True)
        for o, row in zip(outs, rows):
            assert sum(w * q(cpos[c]) for c, w in row.items()) == q(fpos[o])
        outs, rows = op.restriction_rows(face, sub, p, k, 1, exact=True)
        for o, row in zip(outs, rows):
            assert sum(w * q(fpos[c]) for c, w in row.items()) == q(cpos[o])


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("k", [2, 3])
def test_rows_sum_to_one(order, k):
    for face in (0, 4):
        for sub in range(9):
            for build in (op.interpolation_operator, op.restriction_operator):
                _, W = build(face, sub, 9, k, order)
                assert np.abs(np.asarray(W.sum(axis=1)).ravel() - 1).max() < 1e-13


@pytest.mark.parametrize("order", [1, 2, 3])
def test_injection_at_coincident_centres(order):
    # Sec. 3: fine centres that coincide with coarse centres; k > 1 restriction
    # of the first halo layer is an injection
    p, k = 9, 3
    for face in range(6):
        for sub in (0, 4, 7):
            cpos, fpos = _positions(face, sub, p, k)
            outs, rows = op.interpolation_rows(face, sub, p, k, order, exact=True)
            n_coinc = 0
            for o, row in zip(outs, rows):
                if fpos[o] in cpos:
                    n_coinc += 1
                    assert row == {cpos.index(fpos[o]): 1}
            assert n_coinc == (p // 3) ** 2
            if order >= 2:
                outs, rows = op.restriction_rows(face, sub, p, k, order, exact=True)
                n_inj = 0
                for o, row in zip(outs, rows):
                    if cpos[o] in fpos:
                        n_inj += 1
                        assert row == {fpos.index(cpos[o]): 1}
                assert n_inj == (p // 3) ** 2


def _normal_weights(row, face, p, k, t_idx):
    """Weights of a row restricted to one tangential column, keyed by signed
    layer index j (j = -1 is the coarse-side layer next to the interface)."""
    n, t0, t1 = g.axes(face)
    ext = g.extents(face, p, k)
    out = {}
    for col, w in row.items():
        idx = (col % ext[0], (col // ext[0]) % ext[1], col // (ext[0] * ext[1]))
        if (idx[t0], idx[t1]) != t_idx:
            return None
        j = idx[n] - k if face < 3 else k - 1 - idx[n]
        out[j] = w
    return out


def _row_at(outs, rows, face, p, k, normal_j, t_idx):
    n, t0, t1 = g.axes(face)
    ext = g.extents(face, p, k)
    idx = [0, 0, 0]
    idx[n] = normal_j + k if face < 3 else k - 1 - normal_j
    idx[t0], idx[t1] = t_idx
    return rows[outs.index(g.flat(ext, idx))]


@pytest.mark.parametrize("face", [0, 3])
def test_hand_derived_weights(face):
    """Closed-form weights derived by hand from the definitions.

    Signed layers: coarse centre of layer j at (j + 1/2) H, fine layer i at
    (i + 1/2) H/3; negative = coarse side.  Interpolation about coarse layer -1:
      T2, fine layer -1 (offset +H/3), 3-point centred normal stencil on
        layers (-2,-1,0): u + (1/3)(u0 - u-2)/2 + (1/18)(u-2 - 2u-1 + u0)
        = (-1/9, 8/9, 2/9);
      d-linear, fine layer -1: (2/3 on -1, 1/3 on 0); fine layer -3:
        (1/3 on -2, 2/3 on -1).
    Restriction, k = 3, about fine layer 2 (window (0,1,2) clamped inward):
      T2 to coarse layer 1 (offset 2h): u2 + 2u' + 2u'' = (3, -8, 6);
      T2 to coarse layer 2 (offset 5h): u2 + 5u' + 12.5u'' = (15, -35, 21);
      d-linear least-squares line through layers (0,1,2) at 1.5h, 4.5h, 7.5h:
      (1/3, 1/3, 1/3), (-7/6, 1/3, 11/6), (-8/3, 1/3, 10/3)."""
    p, k, sub = 9, 3, 4
    mid = (4, 4)   # fine local column coincident with coarse (4, 4)... in subface 4
    outs, rows = op.interpolation_rows(face, sub, p, k, 2, exact=True)
    # fine local tangential (4,4) of subface 4 is global (13,13) -> coarse (4,4), offset 0
    r = _normal_weights(_row_at(outs, rows, face, p, k, -1, mid), face, p, k, (4, 4))
    assert r == {-2: F(-1, 9), -1: F(8, 9), 0: F(2, 9)}
    outs, rows = op.interpolation_rows(face, sub, p, k, 1, exact=True)
    assert _normal_weights(_row_at(outs, rows, face, p, k, -1, mid), face, p, k, (4, 4)) == {-1: F(2, 3), 0: F(1, 3)}
    assert _normal_weights(_row_at(outs, rows, face, p, k, -3, mid), face, p, k, (4, 4)) == {-2: F(1, 3), -1: F(2, 3)}
    assert _normal_weights(_row_at(outs, rows, face, p, k, -2, mid), face, p, k, (4, 4)) == {-1: 1}
    outs, rows = op.restriction_rows(face, sub, p, k, 2, exact=True)
    # coarse (4,4) lies over subface 4 at fine local (4,4)
    assert _normal_weights(_row_at(outs, rows, face, p, k, 0, (4, 4)), face, p, k, (4, 4)) == {1: 1}
    assert _normal_weights(_row_at(outs, rows, face, p, k, 1, (4, 4)), face, p, k, (4, 4)) == {0: 3, 1: -8, 2: 6}
    assert _normal_weights(_row_at(outs, rows, face, p, k, 2, (4, 4)), face, p, k, (4, 4)) == {0: 15, 1: -35, 2: 21}


def test_hand_derived_dlinear_tangential():
    # at the tangential face boundary there is no coarse neighbour outward (no
    # diagonal data): the fine volume at H/6 extrapolates from coarse centres
    # at H/2 and 3H/2 with weights (4/3, -1/3); interior pattern (1/3, 2/3) |
    # 1 | (2/3, 1/3); tangential restriction averages (1/3, 1/3, 1/3)
    from oracle.operators import dlinear_1d_interpolation
    Mn, M0, M1 = dlinear_1d_interpolation(0, 0, 9, 3)
    assert np.allclose(M0[0, :2], [4 / 3, -1 / 3]) and np.count_nonzero(M0[0]) == 2
    assert np.allclose(M0[3, 0:2], [1 / 3, 2 / 3]) and M0[4, 1] == 1 and np.allclose(M0[5, 1:3], [2 / 3, 1 / 3])
    Mn, M0, M1 = dlinear_1d_interpolation(0, 2, 9, 3)
    assert np.allclose(M0[8, 7:9], [-1 / 3, 4 / 3])


@pytest.mark.parametrize("face", range(6))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_dlinear_tensor_product_equals_assembled_matrix(face, k):
    """Sec. 2: P = Px Py Pz per face; applied axis by axis it equals the single
    assembled sparse matrix."""
    p, U = 6, 3
    rng = np.random.default_rng(7 * face + k)
    ext = g.extents(face, p, k)
    X = rng.standard_normal((ext[2], ext[1], ext[0], U))
    for sub in range(9):
        Y = op.dlinear_tensor_interpolate(face, sub, p, k, X).reshape(-1, U)
        outs, W = op.interpolation_operator(face, sub, p, k, 1)
        assert np.abs(Y[outs] - W @ X.reshape(-1, U)).max() < 1e-14
        mask = np.ones(Y.shape[0], bool)
        mask[outs] = False
        assert np.all(Y[mask] == 0)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("order", [2, 3])
def test_taylor_equals_dlinear_on_linear_data(order, k):
    """Appendix "Testing": the new schemes equal the tensor product on linear
    data for every face configuration."""
    U = 2
    for face in range(6):
        items, cl, fl = wl.make_items([face], [-1], [6], [k], [order], U)
        lin = lambda x: torch.stack([1.5 + 0.3 * x[:, 0] - 0.7 * x[:, 1] + 0.2 * x[:, 2],
                                     -2 + x[:, 0] + x[:, 1] + x[:, 2]], 1)
        coarse, fine = wl.polynomial_buffers(items, U, cl, fl, lin, origins=np.array([[3.0, -2.0, 5.0]]))
        c, f = coarse.numpy(), fine.numpy()
        dl = items.copy()
        dl["order"] = 1
        rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
        assert rel(tr.interpolate(items, U, c, f), tr.interpolate(dl, U, c, f)) < 1e-13
        assert rel(tr.restrict(items, U, f, c), tr.restrict(dl, U, f, c)) < 1e-13


def test_paper_matrix_sizes():
    """Sec. 2: per hanging face P is 9p^2k x 2p^2k and R is p^2k x 18p^2k; one
    call evaluates a 1/9 segment."""
    import scipy.sparse as sp
    for p, k in ((6, 2), (9, 3)):
        P_blocks = [op.interpolation_operator(0, s, p, k, 3)[1] for s in range(9)]
        P = sp.vstack(P_blocks)
        assert P.shape == (9 * p * p * k, 2 * p * p * k)
        R_blocks = [op.restriction_operator(0, s, p, k, 3)[1] for s in range(9)]
        R = sp.block_diag(R_blocks)
        assert R.shape == (p * p * k, 18 * p * p * k)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mirror_equivariance(order):
    """Face f and face f+3 are mirror images along the normal: mirrored input
    gives mirrored output (odd Taylor terms change sign twice)."""
    p, k, U = 6, 3, 2
    rng = np.random.default_rng(order)
    for f in range(3):
        n = f
        ax = 2 - n
        ext = g.extents(f, p, k)
        for sub in (0, 5):
            X = rng.standard_normal((ext[2], ext[1], ext[0], U))
            outs_a, Wa = op.interpolation_operator(f, sub, p, k, order)
            outs_b, Wb = op.interpolation_operator(f + 3, sub, p, k, order)
            Ya = np.zeros((ext[2] * ext[1] * ext[0], U))
            Ya[outs_a] = Wa @ X.reshape(-1, U)
            Yb = np.zeros_like(Ya)
            Yb[outs_b] = Wb @ np.flip(X, ax).reshape(-1, U)
            assert np.abs(np.flip(Ya.reshape(X.shape), ax) - Yb.reshape(X.shape)).max() < 1e-14 * np.abs(Ya).max()
            Ra_o, Ra = op.restriction_operator(f, sub, p, k, order)
            Rb_o, Rb = op.restriction_operator(f + 3, sub, p, k, order)
            Za = np.zeros_like(Ya)
            Za[Ra_o] = Ra @ X.reshape(-1, U)
            Zb = np.zeros_like(Ya)
            Zb[Rb_o] = Rb @ np.flip(X, ax).reshape(-1, U)
            assert np.abs(np.flip(Za.reshape(X.shape), ax) - Zb.reshape(X.shape)).max() < 1e-14 * np.abs(Za).max()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_rotation_equivariance(order):
    """Faces 0 (normal x) and 1 (normal y) share t1 = z; swapping the x and y
    axes of the data maps one configuration onto the other, subface s0 + 3 s1
    onto itself (t0 is y for face 0 and x for face 1)."""
    p, k, U = 6, 2, 1
    rng = np.random.default_rng(11 + order)
    ext0 = g.extents(0, p, k)   # (2k, p, p) as (x, y, z)
    for sub in (1, 3, 4):
        X0 = rng.standard_normal((ext0[2], ext0[1], ext0[0], U))   # (z, y, x, U)
        X1 = np.swapaxes(X0, 1, 2)                                # face-1 array
        outs0, W0 = op.interpolation_operator(0, sub, p, k, order)
        outs1, W1 = op.interpolation_operator(1, sub, p, k, order)
        Y0 = np.zeros((X0.size // U, U))
        Y0[outs0] = W0 @ X0.reshape(-1, U)
        Y1 = np.zeros_like(Y0)
        Y1[outs1] = W1 @ X1.reshape(-1, U)
        assert np.abs(np.swapaxes(Y0.reshape(X0.shape), 1, 2) - Y1.reshape(X1.shape)).max() < 1e-14 * np.abs(Y0).max()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_adjoint_dot_product_identity(order):
    U = 3
    items, cl, fl = wl.make_items([0, 4, 2], [-1, 3, 8], [6, 9, 6], [3, 2, 3], [order] * 3, U)
    rng = np.random.default_rng(order)
    v_c, v_f = rng.standard_normal(cl), rng.standard_normal(fl)
    g_f, g_c = rng.standard_normal(fl), rng.standard_normal(cl)
    Pv = tr.interpolate(items, U, v_c, np.zeros(fl))
    assert abs(np.dot(g_f, Pv) - np.dot(tr.interpolate_adjoint(items, U, g_f, cl), v_c)) < 1e-10
    Rv = tr.restrict(items, U, v_f, np.zeros(cl))
    assert abs(np.dot(g_c, Rv) - np.dot(tr.restrict_adjoint(items, U, g_c, fl), v_f)) < 1e-10


def _smooth(H):
    """exp(a.x) + sin(b.x + c): derivatives of every order are non-zero near
    the limit point, so the leading error term does not vanish there."""
    def f(x):
        x = x * H
        v = (torch.exp(0.7 * x[:, 0] - 0.5 * x[:, 1] + 0.9 * x[:, 2])
             + 0.5 * torch.sin(1.3 * x[:, 0] + 0.4 * x[:, 1] - 0.8 * x[:, 2] + 0.4))
        return v[:, None]
    return f


@pytest.mark.parametrize("face", [1, 3])
@pytest.mark.parametrize("order,expected", [(1, 2.0), (2, 3.0), (3, 4.0)])
def test_convergence_order(order, expected, face):
    """Sec. 5.1: d-linear converges as O(h^2); Taylor-m matches its expansion
    (local error O(H^{m+1}) of the reconstructed values).  Refinement keeps
    the 3:1 ratio and shrinks the face towards a fixed point; the last
    observed max-norm rate must be within 0.3 of the expected order."""
    items, cl, fl = wl.make_items([face], [-1], [9], [3], [order], 1)
    org = np.array([[0.3, -0.2, 0.1]])
    errs_i, errs_r = [], []
    Hs = [0.04 / 2 ** j for j in range(4)]
    for H in Hs:
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
