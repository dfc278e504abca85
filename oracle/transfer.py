"""Buffer-level application of P and R over a list of transfer items
(paper Sec. 2: Q^f = P Q^c per hanging face, Q^c = R Q^f; each call evaluates
the 1/9 block of one subface, Sec. 2 and the appendix "Code Overview").

An item is any mapping with the fields
  face, subface (0..8, or -1 for all nine), patch_size p, overlap k, order,
  coarse_offset, fine_offset, and optionally scheme (0 finite-difference
  derivatives, 1 least-squares fit)
(offsets in float64 elements).  Its coarse face array is
coarse[coarse_offset : coarse_offset + 2k p^2 U]; subface s's fine face array
is fine[fine_offset + j * 2k p^2 U : ...] with j = 0 for a single-subface item
and j = s for a whole-face item.

interpolate  writes only the fine ghost halves;
restrict     writes only the coarse halo volumes over the item's subfaces;
*_adjoint    return the transposed map applied to a gradient, as a fresh
             buffer of the input's size (zeros where no weight reaches),
             summing the contributions of items that share an input array.
"""
import numpy as np

from . import geometry as g
from .operators import interpolation_operator, restriction_operator


def _field(item, name):
    return int(item[name])


def item_subfaces(item):
    """(subface, index of its fine face array within the item) pairs."""
    s = _field(item, "subface")
    return [(j, j) for j in range(9)] if s < 0 else [(s, 0)]


def _geom(item):
    return (_field(item, "face"), _field(item, "patch_size"), _field(item, "overlap"),
            _field(item, "order"))


def _scheme(item):
    """Derivative estimate of a Taylor item: 0 finite differences, 1 least squares."""
    try:
        return int(item["scheme"])
    except (KeyError, ValueError, IndexError):
        return 0


def _arrays(item, U):
    face, p, k, order = _geom(item)
    n = g.face_array_len(p, k) * U
    return n, _field(item, "coarse_offset"), _field(item, "fine_offset")


def interpolate(items, U, coarse, fine):
    """Return a copy of ``fine`` with every item's fine ghost halves set to P coarse."""
    out = np.array(fine, dtype=np.float64, copy=True)
    for item in items:
        face, p, k, order = _geom(item)
        n, co, fo = _arrays(item, U)
        X = np.asarray(coarse[co:co + n], dtype=np.float64).reshape(-1, U)
        for s, j in item_subfaces(item):
            rows, W = interpolation_operator(face, s, p, k, order, _scheme(item))
            view = out[fo + j * n: fo + (j + 1) * n].reshape(-1, U)
            view[rows] = W @ X
    return out


def restrict(items, U, fine, coarse):
    """Return a copy of ``coarse`` with every item's owned coarse halo volumes set to R fine."""
    out = np.array(coarse, dtype=np.float64, copy=True)
    for item in items:
        face, p, k, order = _geom(item)
        n, co, fo = _arrays(item, U)
        view = out[co:co + n].reshape(-1, U)
        for s, j in item_subfaces(item):
            rows, W = restriction_operator(face, s, p, k, order, _scheme(item))
            X = np.asarray(fine[fo + j * n: fo + (j + 1) * n], dtype=np.float64).reshape(-1, U)
            view[rows] = W @ X
    return out


def interpolate_adjoint(items, U, g_fine, coarse_len):
    """P^T applied to the gradient of the fine buffer (only ghost entries count)."""
    out = np.zeros(coarse_len, dtype=np.float64)
    for item in items:
        face, p, k, order = _geom(item)
        n, co, fo = _arrays(item, U)
        acc = out[co:co + n].reshape(-1, U)
        for s, j in item_subfaces(item):
            rows, W = interpolation_operator(face, s, p, k, order, _scheme(item))
            G = np.asarray(g_fine[fo + j * n: fo + (j + 1) * n], dtype=np.float64).reshape(-1, U)
            acc += W.T @ G[rows]
    return out


def restrict_adjoint(items, U, g_coarse, fine_len):
    """R^T applied to the gradient of the coarse buffer (only owned halo entries count)."""
    out = np.zeros(fine_len, dtype=np.float64)
    for item in items:
        face, p, k, order = _geom(item)
        n, co, fo = _arrays(item, U)
        G = np.asarray(g_coarse[co:co + n], dtype=np.float64).reshape(-1, U)
        for s, j in item_subfaces(item):
            rows, W = restriction_operator(face, s, p, k, order, _scheme(item))
            acc = out[fo + j * n: fo + (j + 1) * n].reshape(-1, U)
            acc += W.T @ G[rows]
    return out


def interpolate_one(item, U, coarse, fine_index):
    """P applied for a single output element: fine_index is a flat element
    index of the fine buffer lying in one of the item's ghost halves.  Used to
    check sampled outputs of very large batches one by one."""
    face, p, k, order = _geom(item)
    n, co, fo = _arrays(item, U)
    rel = fine_index - fo
    j, r = divmod(rel, n)
    vol, u = divmod(r, U)
    s = j if _field(item, "subface") < 0 else _field(item, "subface")
    rows, W = interpolation_operator(face, s, p, k, order, _scheme(item))
    rpos = rows.index(vol)
    lo, hi = W.indptr[rpos], W.indptr[rpos + 1]
    cols, vals = W.indices[lo:hi], W.data[lo:hi]
    return float(np.dot(vals, np.asarray(coarse)[co + cols * U + u]))


def restrict_one(item, U, fine, coarse_index):
    """R applied for a single output element of the coarse buffer."""
    face, p, k, order = _geom(item)
    n, co, fo = _arrays(item, U)
    vol, u = divmod(coarse_index - co, U)
    ext = g.extents(face, p, k)
    idx = (vol % ext[0], (vol // ext[0]) % ext[1], vol // (ext[0] * ext[1]))
    _, t0, t1 = g.axes(face)
    s = g.owner_subface_index(idx[t0], p) + 3 * g.owner_subface_index(idx[t1], p)
    j = s if _field(item, "subface") < 0 else 0
    rows, W = restriction_operator(face, s, p, k, order, _scheme(item))
    rpos = rows.index(vol)
    lo, hi = W.indptr[rpos], W.indptr[rpos + 1]
    cols, vals = W.indices[lo:hi], W.data[lo:hi]
    return float(np.dot(vals, np.asarray(fine)[fo + j * n + cols * U + u]))
