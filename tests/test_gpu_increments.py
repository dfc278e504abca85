"""Float32 storage of the interpolation increments (split precision): the
increments against the oracle's (fine ghost value - nearest coarse centre
value), the round trip through apply_increments against the oracle, and
exact zeros at coincident volumes."""
import numpy as np
import pytest
import torch

from oracle import transfer as tr
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import normwise_errors, record, written_masks

pytestmark = pytest.mark.gpu
BOUND = 2e-6


def _reference_increments(items, U, coarse, f_ref):
    """Oracle increments in the documented layout, and the coincidence mask."""
    out, coinc = [], []
    for it in items:
        face, sub, p, k = int(it["face"]), int(it["subface"]), int(it["patch_size"]), int(it["overlap"])
        n = face % 3
        ext = [p, p, p]
        ext[n] = 2 * k
        t0, t1 = [d for d in range(3) if d != n]
        arr = 2 * k * p * p * U
        co, fo = int(it["coarse_offset"]), int(it["fine_offset"])
        subs = list(range(9)) if sub < 0 else [sub]
        for slot, s in enumerate(subs):
            s0, s1 = s % 3, s // 3
            for g in range(k):
                for q1 in range(p):
                    for q0 in range(p):
                        idx = [0, 0, 0]
                        idx[n] = (k - 1 - g) if face < 3 else (k + g)    # fine signed layer -1-g
                        idx[t0], idx[t1] = q0, q1
                        fv = (idx[2] * ext[1] + idx[1]) * ext[0] + idx[0]
                        a, b = (s0 * p + q0) // 3, (s1 * p + q1) // 3
                        cidx = [0, 0, 0]
                        cidx[n] = k - 1 if face < 3 else k               # coarse signed layer -1
                        cidx[t0], cidx[t1] = a, b
                        cv = (cidx[2] * ext[1] + cidx[1]) * ext[0] + cidx[0]
                        fine_vals = f_ref[fo + slot * arr + fv * U: fo + slot * arr + (fv + 1) * U]
                        base = coarse[co + cv * U: co + (cv + 1) * U]
                        out.append(fine_vals - base)
                        coinc.append(np.full(U, g == 1 and (s0 * p + q0) % 3 == 1 and (s1 * p + q1) % 3 == 1))
    return np.concatenate(out), np.concatenate(coinc)


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("precision", [B.PREC_SPLIT, B.PREC_FP64])
def test_increments_and_apply(order, precision):
    U = 9
    faces = [0, 1, 2, 3, 4, 5, 1, 4]
    subs = [-1, -1, -1, -1, -1, -1, 3, 7]
    n = len(faces)
    items, cl, fl = wl.make_items(faces, subs, [9] * 6 + [6, 12], [3] * 6 + [2, 3], [order] * n, U)
    rng = np.random.Generator(np.random.PCG64(55 + order))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(n, rng))
    c, f = coarse.numpy(), fine.numpy()
    plan = B.Plan(items, U, cl, fl, precision)
    ne = plan.info["increment_elems"]
    incr = torch.full((ne,), float("nan"), dtype=torch.float32, device="cuda")
    cd = coarse.cuda()
    plan.interpolate_increments(cd, incr)
    fd = fine.cuda().clone()
    plan.apply_increments(cd, incr, fd)
    torch.cuda.synchronize()
    f_ref = tr.interpolate(items, U, c, f)
    ref_incr, coinc = _reference_increments(items, U, c, f_ref)
    got = incr.cpu().numpy().astype(np.float64)
    assert len(ref_incr) == ne
    assert np.all(got[coinc] == 0.0)
    scale = np.abs(f_ref).max()
    e_incr = np.abs(got - ref_incr).max() / scale
    fmask, _ = written_masks(items, U, cl, fl)
    f_gpu = fd.cpu().numpy()
    assert np.array_equal(f_gpu[~fmask], f[~fmask])
    e_apply, _ = normwise_errors(items, U, f_gpu, f_ref, fmask, "fine")
    record(test="increments", order=order, precision=precision, incr=e_incr, apply=e_apply)
    assert e_incr <= BOUND and e_apply <= BOUND, (e_incr, e_apply)
