"""GPU parity for patch sizes that are not multiples of 3.  Subface boundaries
then cut coarse volumes: the interpolation kernel's CUT variant writes the
children of one coarse centre into two fine face arrays (whole faces) or
drops the ones outside the subface (subface items).  Restriction takes each
coarse halo volume from the subface holding its coincident fine volume,
injecting along a cut axis in the d-linear case.  Compared element by element
with the oracle on the same seeded inputs."""
import numpy as np
import pytest
import torch

from oracle import transfer as tr
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import normwise_errors, record, written_masks
from .test_gpu_increments import BOUND as INCR_BOUND, _reference_increments
from .test_gpu_parity import FP64_TOL, SPLIT_BOUND, _batch, _check

pytestmark = pytest.mark.gpu

PRECISIONS = [(B.PREC_FP64, FP64_TOL), (B.PREC_SPLIT, SPLIT_BOUND), (B.PREC_FIXED, FP64_TOL)]


@pytest.mark.parametrize("precision,tol", PRECISIONS)
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("p,k", [(4, 2), (5, 3), (7, 3), (8, 2), (10, 3), (13, 2)])
def test_whole_faces(p, k, order, precision, tol):
    n = 6
    items, c, f = _batch(list(range(n)), [-1] * n, [p] * n, [k] * n, [order] * n, 11, seed=p * 10 + order)
    _check(items, 11, c, f, precision, tol)


@pytest.mark.parametrize("precision,tol", PRECISIONS)
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("p,k", [(4, 2), (5, 3), (7, 2), (8, 3)])
def test_subface_items(p, k, order, precision, tol):
    faces = [f for f in (0, 4) for _ in range(9)]
    subs = [s for _ in range(2) for s in range(9)]
    n = len(faces)
    items, c, f = _batch(faces, subs, [p] * n, [k] * n, [order] * n, 7, seed=100 + p * 10 + k)
    _check(items, 7, c, f, precision, tol)


def test_dlinear_overlap_one():
    items, c, f = _batch(list(range(6)), [-1] * 6, [5] * 6, [1] * 6, [1] * 6, 3, seed=55)
    _check(items, 3, c, f, B.PREC_FP64, FP64_TOL)


@pytest.mark.parametrize("precision,tol", PRECISIONS)
def test_mixed_patch_sizes_in_one_plan(precision, tol):
    """Multiples of 3 and other sizes together: both interpolation kernel
    variants run in one call; U = 37 splits into unknown chunks.  Two large
    patches (p = 47 and 48) enter as single subfaces."""
    rng = np.random.default_rng(17)
    n = 24
    ps = rng.choice([4, 5, 6, 7, 9, 11, 13], n)
    ks = rng.choice([2, 3], n)
    orders = rng.choice([1, 2, 3], n)
    subs = rng.integers(-1, 9, n)
    ps[:2], ks[:2], orders[:2], subs[:2] = [47, 48], [2, 2], [3, 2], [4, 2]
    items, c, f = _batch(rng.integers(0, 6, n), subs, ps, ks, orders, 37, seed=19)
    _check(items, 37, c, f, precision, tol)
    plan = B.Plan(items, 37, len(c), len(f), precision)
    assert plan.info["interp_launches"] == 2
    plan.close()


@pytest.mark.parametrize("order", [1, 2, 3])
def test_increments_round_trip(order):
    U = 9
    faces, subs = [0, 1, 2, 3, 4, 5, 1, 4], [-1, -1, -1, 5, -1, -1, 3, 7]
    n = len(faces)
    items, cl, fl = wl.make_items(faces, subs, [4, 5, 7, 8, 10, 9, 5, 8], [2, 3, 3, 2, 3, 3, 2, 3], [order] * n, U)
    rng = np.random.Generator(np.random.PCG64(77 + order))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(n, rng))
    c, f = coarse.numpy(), fine.numpy()
    plan = B.Plan(items, U, cl, fl, B.PREC_SPLIT)
    incr = torch.full((plan.info["increment_elems"],), float("nan"), dtype=torch.float32, device="cuda")
    cd = coarse.cuda()
    plan.interpolate_increments(cd, incr)
    fd = fine.cuda().clone()
    plan.apply_increments(cd, incr, fd)
    torch.cuda.synchronize()
    f_ref = tr.interpolate(items, U, c, f)
    ref_incr, coinc = _reference_increments(items, U, c, f_ref)
    got = incr.cpu().numpy().astype(np.float64)
    assert not np.isnan(got).any()
    assert np.all(got[coinc] == 0.0)
    e_incr = np.abs(got - ref_incr).max() / np.abs(f_ref).max()
    fmask, _ = written_masks(items, U, cl, fl)
    f_gpu = fd.cpu().numpy()
    assert np.array_equal(f_gpu[~fmask], f[~fmask])
    e_apply, _ = normwise_errors(items, U, f_gpu, f_ref, fmask, "fine")
    record(test="increments_general_p", order=order, incr=e_incr, apply=e_apply)
    assert e_incr <= INCR_BOUND and e_apply <= INCR_BOUND, (e_incr, e_apply)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_adjoints_match_oracle_transposes(order):
    U = 5
    p, k = 7, 3
    arr = 2 * k * p * p * U
    items = np.zeros(9 + 3, dtype=wl.ITEM_DTYPE)
    for s in range(9):  # nine subfaces sharing one coarse face array
        items[s] = (1, s, p, k, order, 0, 0, s * arr)
    for j, (f, pp) in enumerate(((0, 4), (3, 8), (5, 5))):
        items[9 + j] = (f, -1, pp, k, order, 0, arr + j * 2 * 8 * 8 * k * U, 9 * arr + j * 9 * 2 * 8 * 8 * k * U)
    cl, fl = arr + 3 * 2 * 8 * 8 * k * U, 9 * arr + 3 * 9 * 2 * 8 * 8 * k * U
    rng = np.random.default_rng(order)
    g_f, g_c = rng.standard_normal(fl), rng.standard_normal(cl)
    plan = B.Plan(items, U, cl, fl, B.PREC_FP64)
    out_c = torch.full((cl,), np.nan, dtype=torch.float64, device="cuda")
    plan.interpolate_adjoint(torch.as_tensor(g_f).cuda(), out_c)
    out_f = torch.full((fl,), np.nan, dtype=torch.float64, device="cuda")
    plan.restrict_adjoint(torch.as_tensor(g_c).cuda(), out_f)
    torch.cuda.synchronize()
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    e1 = rel(out_c.cpu().numpy(), tr.interpolate_adjoint(items, U, g_f, cl))
    e2 = rel(out_f.cpu().numpy(), tr.restrict_adjoint(items, U, g_c, fl))
    record(test="adjoint_general_p", order=order, pt=e1, rt=e2)
    assert e1 <= FP64_TOL and e2 <= FP64_TOL, (e1, e2)


@pytest.mark.parametrize("scheme,flags", [(1, 0), (0, B.FLAG_CSR)])
def test_least_squares_and_sparse_row_kernels(scheme, flags):
    """The least-squares scheme (factorised kernels, CUT variant for these
    patch sizes) and AMR_FLAG_CSR (sparse-row kernels, whose rows the host
    builds for any patch size)."""
    n = 8
    orders = [3, 2, 3, 2, 3, 2, 3, 2] if scheme else [1, 2, 3, 1, 2, 3, 1, 2]
    items, c, f = _batch(list(range(6)) + [2, 5], [-1, 4, -1, 0, 8, -1, 3, -1], [4, 5, 7, 8, 10, 5, 7, 4],
                         [2, 3, 3, 2, 3, 2, 3, 3], orders, 7, seed=200 + scheme)
    items["scheme"] = scheme
    plan = B.Plan(items, 7, len(c), len(f), B.PREC_FP64, flags)
    fm, cm = written_masks(items, 7, len(c), len(f))
    from .parity import gpu_interpolate, gpu_restrict
    f_gpu = gpu_interpolate(plan, c, f)
    assert np.array_equal(f_gpu[~fm], f[~fm])
    e_i = normwise_errors(items, 7, f_gpu, tr.interpolate(items, 7, c, f), fm, "fine")[0]
    c_gpu = gpu_restrict(plan, f, c)
    assert np.array_equal(c_gpu[~cm], c[~cm])
    e_r = normwise_errors(items, 7, c_gpu, tr.restrict(items, 7, f, c), cm, "coarse")[0]
    record(test="sparse_rows_general_p", scheme=scheme, interp=e_i, restrict=e_r)
    assert e_i <= FP64_TOL and e_r <= FP64_TOL, (e_i, e_r)
