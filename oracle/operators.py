"""Operator rows of P (interpolation) and R (restriction), one output volume
at a time, in the face's physical frame.

Taylor-m (m = 2, 3), paper Sec. 3:
  interpolation  per fine ghost volume f: the nearest coarse centre c (unique
                 under three-partitioning); derivatives D^alpha u(c),
                 0 < |alpha| <= m, from tensor finite-difference stencils over
                 the coarse face array; u(f) = sum_alpha D^alpha u(c)
                 (x_f - x_c)^alpha / alpha!.
  restriction    per coarse halo volume C: the nearest fine volume f* of the
                 subface's fine face array (coincident when k > 1 and C is in
                 the first halo layer: injection); derivatives at f* on the
                 fine grid; Taylor's formula to x_C (extrapolation otherwise).
d-linear (order 1), paper Sec. 2:
  interpolation  per axis, linear Lagrange interpolation between the two
                 coarse centres that bracket the fine centre (extrapolation from
                 the two nearest where no bracketing pair exists, i.e. at the
                 tangential face boundary); the operator is the tensor product.
  restriction    tangentially the average of the 3 fine volumes inside the
                 coarse volume; normally the least-squares line through the
                 fine patch's own layers (plus the adjacent ghost layer when
                 k = 1) evaluated at the coarse centre; tensor product.

Rows are dicts {column: weight} over the flat volume indices of the input
face array.  ``exact=True`` keeps every weight a Fraction; otherwise the
exact 1-D weights are rounded to float once and combined in float64.
"""
from fractions import Fraction
from functools import lru_cache
from itertools import product

from . import geometry as g
from .stencils import (Unsupported, exactness_degree, lagrange_derivative_weights,
                       multi_indices, window)

ORDER_DLINEAR, ORDER_TAYLOR2, ORDER_TAYLOR3 = 1, 2, 3
SCHEME_FD, SCHEME_LS = 0, 1


def _factorial(n):
    out = 1
    for r in range(2, n + 1):
        out *= r
    return out


def _nearest(target, candidates):
    """Index into candidates of the point nearest to target; asserts uniqueness.

    Every cell centre is a multiple of H/6, so squared distances are compared
    exactly on integer coordinates scaled by 6."""
    import numpy as np
    cand = np.array([[int(c * 6) for c in x] for x in candidates], dtype=np.int64) \
        if not isinstance(candidates, np.ndarray) else candidates
    t = np.array([int(c * 6) for c in target], dtype=np.int64)
    d2 = ((cand - t) ** 2).sum(axis=1)
    order = np.argsort(d2, kind="stable")
    if len(order) > 1 and d2[order[0]] == d2[order[1]]:
        raise AssertionError("nearest cell is not unique")
    return int(order[0])


def _scaled(points):
    """Centres as an int64 array scaled by 6 (exact)."""
    import numpy as np
    out = np.array([[int(c * 6) for c in x] for x in points], dtype=np.int64)
    assert all(Fraction(int(c * 6)) == c * 6 for x in points for c in x)
    return out


def _axis_stencil(centre_idx, extent, alpha_d, E_d, num):
    """1-D stencil {index: weight} of the alpha_d-th derivative at centre_idx
    along an axis holding indices [0, extent) at unit spacing."""
    if alpha_d == 0:
        return {centre_idx: num(1)}
    pts = window(centre_idx, 0, extent - 1, E_d)
    w = lagrange_derivative_weights(tuple(q - centre_idx for q in pts), 0, alpha_d)
    return {q: num(wq) for q, wq in zip(pts, w) if wq != 0}


def taylor_row(centre_idx, ext, offset, order, num):
    """Row of the Taylor-m reconstruction about centre_idx evaluated at
    ``offset`` (x_out - x_centre, in units of the input grid spacing).

    u(out) = sum_{|alpha| <= m} D^alpha u(centre) offset^alpha / alpha!, with
    D^alpha the tensor product of the per-axis stencils."""
    row = {}
    for alpha in multi_indices(order):
        coeff = Fraction(1)
        for d in range(3):
            coeff *= Fraction(offset[d]) ** alpha[d] / _factorial(alpha[d])
        if coeff == 0:
            continue
        axis_st = [
            _axis_stencil(centre_idx[d], ext[d], alpha[d], exactness_degree(alpha, d, order), num)
            for d in range(3)
        ]
        c = num(coeff)
        for (i0, w0), (i1, w1), (i2, w2) in product(*(sorted(s.items()) for s in axis_st)):
            col = g.flat(ext, (i0, i1, i2))
            row[col] = row.get(col, num(0)) + c * w0 * w1 * w2
    return row


def _stencil_support(centre_idx, ext, order):
    """Every centre the tensor stencils of the derivatives 0 < |alpha| <= m
    touch (the union of their windows), as index triples."""
    pts = set()
    for alpha in multi_indices(order):
        if sum(alpha) == 0:
            continue
        axes = []
        for d in range(3):
            if alpha[d] == 0:
                axes.append((centre_idx[d],))
            else:
                axes.append(window(centre_idx[d], 0, ext[d] - 1, exactness_degree(alpha, d, order)))
        pts.update(product(*axes))
    return sorted(pts)


def _solve(M, B):
    """Exact solution X of M X = B (Fractions, Gauss-Jordan with pivoting)."""
    n = len(M)
    aug = [list(M[i]) + list(B[i]) for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        inv = 1 / aug[col][col]
        aug[col] = [v * inv for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [a - f * b for a, b in zip(aug[r], aug[col])]
    return [row[n:] for row in aug]


@lru_cache(maxsize=None)
def _ls_derivative_weights(rel_points, order):
    """Least-squares fit of the derivatives D^alpha (0 < |alpha| <= m) to the
    differences u_j - u_c at the points rel_points (offsets from the centre,
    grid units): the basis of alpha at offset r is r^alpha / alpha!, the
    fitted x = (A^T A)^-1 A^T (u - u_c).  Returns {alpha: [weight per point]}."""
    alphas = [a for a in multi_indices(order) if sum(a) > 0]
    A = []
    for r in rel_points:
        A.append([F_prod([Fraction(r[d]) ** a[d] / _factorial(a[d]) for d in range(3)]) for a in alphas])
    # derivatives the points carry no information about (a zero column: e.g.
    # tangential ones for points on one normal line) are not fitted
    keep = [i for i in range(len(alphas)) if any(row[i] != 0 for row in A)]
    alphas = [alphas[i] for i in keep]
    A = [[row[i] for i in keep] for row in A]
    n = len(alphas)
    AtA = [[sum(A[i][p] * A[i][q] for i in range(len(A))) for q in range(n)] for p in range(n)]
    At = [[A[i][p] for i in range(len(A))] for p in range(n)]
    G = _solve(AtA, At)
    return {a: G[i] for i, a in enumerate(alphas)}


def F_prod(vals):
    out = Fraction(1)
    for v in vals:
        out *= v
    return out


def taylor_ls_row(centre_idx, ext, offset, order, num, points=None):
    """Row of the least-squares Taylor-m reconstruction (paper Sec. 3: a
    polynomial fit through neighbouring centres, A x = Q^c, solved in the
    least-squares sense) about centre_idx, evaluated at ``offset``.  The fit
    passes through the centre value; the points are the FD stencils' support
    (or ``points``)."""
    c = tuple(centre_idx)
    pts = [q for q in (points if points is not None else _stencil_support(c, ext, order)) if tuple(q) != c]
    rel = tuple(tuple(q[d] - c[d] for d in range(3)) for q in pts)
    G = _ls_derivative_weights(rel, order)
    for alpha in multi_indices(order):
        if sum(alpha) > 0 and alpha not in G:  # not fitted: its Taylor term must vanish here
            assert F_prod([Fraction(offset[d]) ** alpha[d] for d in range(3)]) == 0
    w = [Fraction(0)] * len(pts)
    for alpha, g in G.items():
        coeff = F_prod([Fraction(offset[d]) ** alpha[d] / _factorial(alpha[d]) for d in range(3)])
        if coeff == 0:
            continue
        for i in range(len(pts)):
            w[i] += coeff * g[i]
    row = {}
    for q, wi in zip(pts, w):
        if wi != 0:
            row[g_flat(ext, q)] = num(wi)
    row[g_flat(ext, c)] = num(1 - sum(w))
    return row


def g_flat(ext, idx):
    return g.flat(ext, idx)


def _bracket_weights(coords, x, num):
    """Linear Lagrange weights {index: weight} at x from the two entries of the
    sorted coordinate list that bracket x (the two nearest at either end)."""
    for i, c in enumerate(coords):
        if c == x:
            return {i: num(1)}
    if x < coords[0]:
        lo = 0
    elif x > coords[-1]:
        lo = len(coords) - 2
    else:
        lo = max(i for i, c in enumerate(coords) if c < x)
    x0, x1 = coords[lo], coords[lo + 1]
    return {lo: num((x1 - x) / (x1 - x0)), lo + 1: num((x - x0) / (x1 - x0))}


def _ls_line_weights(coords, x, num):
    """Weights of the least-squares line through (coords[i], u_i) at x."""
    nn = len(coords)
    mean = sum(coords) / nn
    sxx = sum((c - mean) ** 2 for c in coords)
    return [num(Fraction(1, nn) + (c - mean) * (x - mean) / sxx) for c in coords]


def _outer_row(ext, axis_weights, num):
    row = {}
    for (i0, w0), (i1, w1), (i2, w2) in product(*(sorted(a.items()) for a in axis_weights)):
        col = g.flat(ext, (i0, i1, i2))
        row[col] = row.get(col, num(0)) + w0 * w1 * w2
    return row


def _num(exact):
    return (lambda v: Fraction(v)) if exact else (lambda v: float(v))


def interpolation_rows(face, sub, p, k, order, exact=False, scheme=SCHEME_FD):
    """Rows of P for subface ``sub``: (output volumes of the fine face array,
    rows over the coarse face array).  Outputs are the fine ghost volumes in
    flat order.  scheme: SCHEME_FD (tensor finite-difference derivatives) or
    SCHEME_LS (least-squares fit of all derivatives at once)."""
    num = _num(exact)
    ext = g.extents(face, p, k)
    coarse_idx = g.all_indices(ext)
    coarse_x = [g.coarse_centre(face, p, k, idx) for idx in coarse_idx]
    coarse_s = _scaled(coarse_x)
    outs, rows = [], []
    for fidx in g.fine_ghost_indices(face, p, k):
        xf = g.fine_centre(face, p, k, sub, fidx)
        if order == ORDER_DLINEAR:
            axis_w = []
            for d in range(3):
                coords = sorted({x[d] for x in coarse_x})
                axis_w.append(_bracket_weights(coords, xf[d], num))
            row = _outer_row(ext, axis_w, num)
        else:
            ci = _nearest(xf, coarse_s)
            xc = coarse_x[ci]
            off = [xf[d] - xc[d] for d in range(3)]
            if scheme == SCHEME_LS:
                row = taylor_ls_row(coarse_idx[ci], ext, off, order, num)
            else:
                row = taylor_row(coarse_idx[ci], ext, off, order, num)
        outs.append(g.flat(ext, fidx))
        rows.append(row)
    return outs, rows


def diagonal_ghost_indices(face, p, k):
    """Extended (diagonal) ghost volumes of one subface: the coarse-side
    layers of the fine face array's index box widened tangentially by k on
    each side, minus the ordinary ghost half -- tangential indices in
    [-k, p + k) with at least one outside [0, p).  Returned as index triples
    in the face array's axis order (they address positions, not storage)."""
    n, t0, t1 = g.axes(face)
    ghost_layers = sorted({idx[n] for idx in g.fine_ghost_indices(face, p, k)})
    out = []
    for i in ghost_layers:
        for b in range(-k, p + k):
            for a in range(-k, p + k):
                if 0 <= a < p and 0 <= b < p:
                    continue
                idx = [0, 0, 0]
                idx[n], idx[t0], idx[t1] = i, a, b
                out.append(tuple(idx))
    return out


def diagonal_interpolation_rows(face, sub, p, k, order, exact=False):
    """Rows of the diagonal-halo interpolation of subface ``sub`` (a reading:
    the paper has no diagonal data, Sec. 2): every extended ghost volume
    (diagonal_ghost_indices) is reconstructed from the coarse face array by
    the same rule as the ordinary ghost volumes -- Taylor-m about the nearest
    coarse centre of the face array (on the face's edge when the volume lies
    past it, the offset then exceeding H/3), with that centre's stencils; or
    the d-linear tensor product with linear extrapolation past the edge.
    Returns (index triples, rows over the coarse face array)."""
    num = _num(exact)
    ext = g.extents(face, p, k)
    coarse_idx = g.all_indices(ext)
    coarse_x = [g.coarse_centre(face, p, k, idx) for idx in coarse_idx]
    coarse_s = _scaled(coarse_x)
    outs, rows = [], []
    for fidx in diagonal_ghost_indices(face, p, k):
        xf = g.fine_centre(face, p, k, sub, fidx)
        if order == ORDER_DLINEAR:
            axis_w = []
            for d in range(3):
                coords = sorted({x[d] for x in coarse_x})
                axis_w.append(_bracket_weights(coords, xf[d], num))
            row = _outer_row(ext, axis_w, num)
        else:
            ci = _nearest(xf, coarse_s)
            xc = coarse_x[ci]
            row = taylor_row(coarse_idx[ci], ext, [xf[d] - xc[d] for d in range(3)], order, num)
        outs.append(fidx)
        rows.append(row)
    return outs, rows


def restriction_rows(face, sub, p, k, order, exact=False, scheme=SCHEME_FD):
    """Rows of R for subface ``sub``: (output volumes of the coarse face array,
    rows over subface sub's fine face array).  With SCHEME_LS the fit uses the
    fine centres on the normal line through the expansion cell (the only
    direction with a non-zero offset), inside the FD normal window."""
    num = _num(exact)
    n = g.axes(face)[0]
    side = g.coarse_side(face)
    ext = g.extents(face, p, k)
    fine_idx = g.all_indices(ext)
    fine_x = [g.fine_centre(face, p, k, sub, idx) for idx in fine_idx]
    fine_s = _scaled(fine_x)
    outs, rows = [], []
    for cidx in g.coarse_halo_indices(face, p, k, sub):
        xC = g.coarse_centre(face, p, k, cidx)
        if order == ORDER_DLINEAR:
            axis_w = []
            for d in range(3):
                coords = [(i - k + Fraction(1, 2)) / 3 if d == n else None for i in range(ext[d])]
                if d == n:
                    # the fine patch's own layers, plus the adjacent ghost layer if k == 1
                    own = [i for i in range(ext[d]) if coords[i] * side < 0]
                    if len(own) < 2:
                        adj = min((i for i in range(ext[d]) if coords[i] * side > 0),
                                  key=lambda i: abs(coords[i]))
                        own = sorted(own + [adj])
                    lw = _ls_line_weights([coords[i] for i in own], xC[d], num)
                    axis_w.append(dict(zip(own, lw)))
                else:
                    # least-squares line through the subface's fine volumes
                    # inside the coarse volume, at its centre: the average of
                    # all three, or the coincident one if a subface boundary
                    # cuts the coarse volume (p not a multiple of 3)
                    inside = [i for i in range(ext[d])
                              if abs(fine_x[g.flat(ext, _unit(d, i))][d] - xC[d]) < Fraction(1, 2)]
                    xs = [fine_x[g.flat(ext, _unit(d, i))][d] for i in inside]
                    axis_w.append(dict(zip(inside, _ls_line_weights(xs, xC[d], num))))
            row = _outer_row(ext, axis_w, num)
        else:
            fi = _nearest(xC, fine_s)
            xf = fine_x[fi]
            offset = [(xC[d] - xf[d]) * 3 for d in range(3)]  # in units of h
            if scheme == SCHEME_LS:
                fidx = fine_idx[fi]
                line = window(fidx[n], 0, ext[n] - 1, order)
                pts = []
                for q in line:
                    idx = list(fidx)
                    idx[n] = q
                    pts.append(tuple(idx))
                row = taylor_ls_row(fidx, ext, offset, order, num, points=pts)
            else:
                row = taylor_row(fine_idx[fi], ext, offset, order, num)
        outs.append(g.flat(ext, cidx))
        rows.append(row)
    return outs, rows


def _unit(d, i):
    idx = [0, 0, 0]
    idx[d] = i
    return tuple(idx)


def check_supported(p, k, order, scheme=SCHEME_FD):
    """Raise Unsupported for combinations the reading cannot serve."""
    if p < 3:
        raise Unsupported(f"patch size {p} must be at least 3")
    if k < 1 or k > p:
        raise Unsupported(f"overlap {k} must satisfy 1 <= k <= p")
    if order not in (ORDER_DLINEAR, ORDER_TAYLOR2, ORDER_TAYLOR3):
        raise Unsupported(f"order {order}")
    if order >= 2 and (2 * k < order + 1 or p < order + 1):
        raise Unsupported(f"Taylor-{order} needs 2k >= {order + 1} and p >= {order + 1}")
    if scheme not in (SCHEME_FD, SCHEME_LS) or (scheme == SCHEME_LS and order == ORDER_DLINEAR):
        raise Unsupported(f"scheme {scheme} with order {order}")


@lru_cache(maxsize=None)
def interpolation_operator(face, sub, p, k, order, scheme=SCHEME_FD):
    """(output flat indices, scipy CSR matrix) of P for one subface, float64."""
    check_supported(p, k, order, scheme)
    outs, rows = interpolation_rows(face, sub, p, k, order, scheme=scheme)
    return outs, _csr(rows, g.face_array_len(p, k))


@lru_cache(maxsize=None)
def restriction_operator(face, sub, p, k, order, scheme=SCHEME_FD):
    """(output flat indices, scipy CSR matrix) of R for one subface, float64."""
    check_supported(p, k, order, scheme)
    outs, rows = restriction_rows(face, sub, p, k, order, scheme=scheme)
    return outs, _csr(rows, g.face_array_len(p, k))


def _csr(rows, ncols):
    import numpy as np
    import scipy.sparse as sp
    indptr, indices, data = [0], [], []
    for row in rows:
        for col in sorted(row):
            indices.append(col)
            data.append(float(row[col]))
        indptr.append(len(indices))
    return sp.csr_matrix((np.array(data, dtype=np.float64), np.array(indices, dtype=np.int64),
                          np.array(indptr, dtype=np.int64)), shape=(len(rows), ncols))


# ---------------------------------------------------------------------------
# d-linear as a tensor product of 1-D operators (paper Sec. 2: P = Px Py Pz,
# P_perp along the normal, P_par applied twice along the tangential axes).
# ---------------------------------------------------------------------------

def dlinear_1d_interpolation(face, sub, p, k):
    """(M_n, M_t0, M_t1) as float64 arrays: M_n maps the 2k coarse layers to
    the fine array's 2k layers (zero rows on the fine patch's own side), M_t
    maps p coarse tangential volumes to the subface's p fine volumes."""
    import numpy as np
    n, t0, t1 = g.axes(face)
    s = g.subface_pos(face, sub)
    side = g.coarse_side(face)
    half = Fraction(1, 2)
    cn = [Fraction(i - k) + half for i in range(2 * k)]
    Mn = np.zeros((2 * k, 2 * k))
    for i in range(2 * k):
        xf = (Fraction(i - k) + half) / 3
        if xf * side > 0:
            for j, w in _bracket_weights(cn, xf, float).items():
                Mn[i, j] = w
    Mt = []
    ct = [Fraction(a) + half for a in range(p)]
    for st in s:
        M = np.zeros((p, p))
        for q in range(p):
            xf = (Fraction(st * p + q) + half) / 3
            for a, w in _bracket_weights(ct, xf, float).items():
                M[q, a] = w
        Mt.append(M)
    return Mn, Mt[0], Mt[1]


def dlinear_tensor_interpolate(face, sub, p, k, coarse_face):
    """Apply P = P_t1 P_t0 P_n to one coarse face array, shaped
    (E_z, E_y, E_x, U) (x fastest), one axis after the other; returns the
    whole fine face array (zeros outside the ghost half)."""
    import numpy as np
    n, t0, t1 = g.axes(face)
    Mn, M0, M1 = dlinear_1d_interpolation(face, sub, p, k)
    mats = {n: Mn, t0: M0, t1: M1}
    out = coarse_face
    for d in (n, t0, t1):
        ax = 2 - d  # array axis of spatial axis d in (z, y, x, U) order
        out = np.moveaxis(np.tensordot(mats[d], out, axes=([1], [ax])), 0, ax)
    return out
