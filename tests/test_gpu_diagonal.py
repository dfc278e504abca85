"""GPU parity of the diagonal (edge and vertex) ghost volumes against the
oracle (a reading: the paper exchanges no diagonal data, Sec. 2).  Every
widened ghost box of every fine face array: the volumes outside the subface
against the oracle's diagonal rows, the volumes inside against its ordinary
interpolation; float64, 1e-12 normwise per (item, unknown)."""
import numpy as np
import pytest
import torch

from oracle import geometry as g
from oracle import operators as op
from oracle import transfer as tr
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import record

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _batch(faces, subs, ps, ks, orders, U, seed):
    items, cl, fl = wl.make_items(faces, subs, ps, ks, orders, U)
    rng = np.random.Generator(np.random.PCG64(wl.SEED_BASE + 300 + seed))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(len(items), rng))
    return items, coarse.numpy(), fine.numpy()


def _expected(items, U, coarse, fine):
    """(expected, mask of positions checked) in the diagonal layout."""
    f_ref = tr.interpolate(items, U, coarse, fine)
    n = B.diagonal_elems(items, U)
    exp = np.full(n, np.nan)
    off = 0
    for it in items:
        face, p, k, m = int(it["face"]), int(it["patch_size"]), int(it["overlap"]), int(it["order"])
        nmain, t0, t1 = g.axes(face)
        ext = g.extents(face, p, k)
        W = p + 2 * k
        co, fo = int(it["coarse_offset"]), int(it["fine_offset"])
        arr = 2 * k * p * p * U
        subs = range(9) if int(it["subface"]) < 0 else [int(it["subface"])]
        c_arr = coarse[co:co + arr].reshape(-1, U)
        for slot, sub in enumerate(subs):
            base = off + slot * k * W * W * U

            def put(idx, vals):
                i_n = idx[nmain]
                gl = k - 1 - i_n if face < 3 else i_n - k
                pos = (gl * W + idx[t1] + k) * W + idx[t0] + k
                exp[base + pos * U:base + (pos + 1) * U] = vals

            outs, rows = op.diagonal_interpolation_rows(face, sub, p, k, m)
            for idx, row in zip(outs, rows):
                cols = np.fromiter(row.keys(), dtype=np.int64)
                w = np.fromiter(row.values(), dtype=np.float64)
                put(idx, w @ c_arr[cols])
            f_arr = f_ref[fo + slot * arr:fo + (slot + 1) * arr].reshape(-1, U)
            for idx in g.fine_ghost_indices(face, p, k):
                put(idx, f_arr[g.flat(ext, idx)])
        off += len(subs) * k * W * W * U
    assert not np.isnan(exp).any()
    return exp


CASES = [
    # faces, subfaces, p, k, order
    ([0, 1, 2, 3, 4, 5], [-1, 0, 4, 8, 2, -1], [6, 9, 6, 9, 7, 6], [3, 2, 3, 3, 2, 2], 3),
    ([0, 1, 2, 3, 4, 5], [-1, 0, 4, 8, 2, -1], [6, 9, 6, 9, 7, 6], [2, 3, 3, 2, 3, 2], 2),
    ([0, 1, 2, 3, 4, 5], [-1, 0, 4, 8, 2, -1], [6, 9, 6, 9, 7, 6], [1, 2, 3, 3, 2, 1], 1),
]


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_FIXED])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_diagonal_halos_match_oracle(case, precision):
    faces, subs, ps, ks, order = CASES[case]
    U = 5
    items, c, f = _batch(faces, subs, ps, ks, [order] * len(faces), U, seed=case)
    exp = _expected(items, U, c, f)
    plan = B.Plan(items, U, len(c), len(f), precision)
    diag = torch.full((plan.diagonal_elems,), float("nan"), dtype=torch.float64, device="cuda")
    plan.interpolate_diagonal(torch.as_tensor(c).cuda(), diag)
    torch.cuda.synchronize()
    got = diag.cpu().numpy()
    plan.close()
    # normwise per (item, unknown) over the item's widened boxes
    worst, off = 0.0, 0
    for it in items:
        p, k = int(it["patch_size"]), int(it["overlap"])
        n = (9 if int(it["subface"]) < 0 else 1) * k * (p + 2 * k) ** 2 * U
        gi, ei = got[off:off + n].reshape(-1, U), exp[off:off + n].reshape(-1, U)
        err = np.abs(gi - ei).max(axis=0) / np.maximum(np.abs(ei).max(axis=0), 1e-300)
        worst = max(worst, float(err.max()))
        off += n
    record(test="diagonal", case=case, order=order, precision=precision, worst=worst)
    assert worst <= TOL, worst


def test_diagonal_rejects_short_buffer_and_deep_overlap():
    U = 2
    items, c, f = _batch([0], [-1], [6], [3], [3], U, seed=9)
    plan = B.Plan(items, U, len(c), len(f), B.PREC_FP64)
    n = plan.diagonal_elems
    short = torch.zeros(n - 1, dtype=torch.float64, device="cuda")
    st = B.lib().amr_transfer_plan_interpolate_diagonal(plan._handle, torch.as_tensor(c).cuda().data_ptr(),
                                                        short.data_ptr(), n - 1, None)
    assert st == 1
    plan.close()
    items, c, f = _batch([2], [4], [9], [4], [3], U, seed=10)
    plan = B.Plan(items, U, len(c), len(f), B.PREC_FP64)
    diag = torch.zeros(plan.diagonal_elems, dtype=torch.float64, device="cuda")
    st = B.lib().amr_transfer_plan_interpolate_diagonal(plan._handle, torch.as_tensor(c).cuda().data_ptr(),
                                                        diag.data_ptr(), plan.diagonal_elems, None)
    assert st == 2
    plan.close()
