"""GPU parity of the least-squares scheme (paper Sec. 3 read as a
least-squares polynomial fit; the factorised kernels with per-class fit
tables) and of the sparse-row (CSR) kernels that serve every item under
AMR_FLAG_CSR, against the oracle."""
import numpy as np
import pytest
import torch

from oracle import transfer as tr
from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

from .parity import gpu_interpolate, gpu_restrict, normwise_errors, record, written_masks

pytestmark = pytest.mark.gpu


def _batch(orders, schemes, U=7, seed=3):
    n = len(orders)
    faces = [i % 6 for i in range(n)]
    subs = [-1 if i % 3 == 0 else (i * 5) % 9 for i in range(n)]
    ps = [9 if i % 2 == 0 else 6 for i in range(n)]
    ks = [3 if i % 4 < 2 else 2 for i in range(n)]
    items, cl, fl = wl.make_items(faces, subs, ps, ks, orders, U)
    items["scheme"] = schemes
    rng = np.random.Generator(np.random.PCG64(wl.SEED_BASE + 300 + seed))
    coarse, fine = wl.sample_buffers(items, U, cl, fl, wl.SmoothField(U, rng), wl.origins_in_box(n, rng))
    return items, coarse.numpy(), fine.numpy()


def _check(items, U, c, f, precision, tol_i, tol_r, flags=0, tag=""):
    plan = B.Plan(items, U, len(c), len(f), precision, flags)
    fm, cm = written_masks(items, U, len(c), len(f))
    f_gpu = gpu_interpolate(plan, c, f)
    assert np.array_equal(f_gpu[~fm], f[~fm])
    e_i = normwise_errors(items, U, f_gpu, tr.interpolate(items, U, c, f), fm, "fine")[0]
    c_gpu = gpu_restrict(plan, f, c)
    assert np.array_equal(c_gpu[~cm], c[~cm])
    e_r = normwise_errors(items, U, c_gpu, tr.restrict(items, U, f, c), cm, "coarse")[0]
    record(test="schemes", tag=tag, precision=precision, interp=e_i, restrict=e_r)
    assert e_i <= tol_i and e_r <= tol_r, (e_i, e_r)
    return plan


# Split-precision restriction: injection, one float64 layer and float-pair
# deeper layers, so its error stays near 2^-44 of sum |w_i| |u_i - u_base|.
SPLIT_RESTRICT_TOL = 1e-10


@pytest.mark.parametrize("precision,tol_i,tol_r", [(B.PREC_FP64, 1e-12, 1e-12),
                                                   (B.PREC_SPLIT, 2e-6, SPLIT_RESTRICT_TOL)])
@pytest.mark.parametrize("order", [2, 3])
def test_least_squares_items(order, precision, tol_i, tol_r):
    items, c, f = _batch([order] * 12, [1] * 12)
    _check(items, 7, c, f, precision, tol_i, tol_r, tag=f"ls{order}")


def test_mixed_fd_and_ls_items_in_one_plan():
    orders = [3, 2, 3, 1, 2, 3, 1, 3, 2, 2, 3, 1]
    schemes = [1, 0, 0, 0, 1, 1, 0, 0, 0, 1, 1, 0]
    items, c, f = _batch(orders, schemes, seed=8)
    _check(items, 7, c, f, B.PREC_FP64, 1e-12, 1e-12, tag="mixed")


@pytest.mark.parametrize("precision,tol_i", [(B.PREC_FP64, 1e-12), (B.PREC_SPLIT, 2e-6), (B.PREC_FIXED, 1e-12)])
@pytest.mark.parametrize("order", [1, 2, 3])
def test_csr_flag_reproduces_factorised_operators(order, precision, tol_i):
    items, c, f = _batch([order] * 12, [0] * 12, seed=11)
    plan = _check(items, 7, c, f, precision, tol_i, 1e-12, flags=B.FLAG_CSR, tag=f"csr{order}")
    assert plan.info["interp_launches"] == 1


def test_least_squares_adjoint_matches_oracle_transposes():
    U = 5
    items, c, f = _batch([3, 2, 3, 2, 3, 3], [1] * 6, U=U, seed=21)
    plan = B.Plan(items, U, len(c), len(f), B.PREC_FP64)
    rng = np.random.default_rng(4)
    gf, gc = rng.standard_normal(len(f)), rng.standard_normal(len(c))
    oc = torch.empty(len(c), dtype=torch.float64, device="cuda")
    of = torch.empty(len(f), dtype=torch.float64, device="cuda")
    plan.interpolate_adjoint(torch.as_tensor(gf).cuda(), oc)
    plan.restrict_adjoint(torch.as_tensor(gc).cuda(), of)
    torch.cuda.synchronize()
    ref_c = tr.interpolate_adjoint(items, U, gf, len(c))
    ref_f = tr.restrict_adjoint(items, U, gc, len(f))
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(oc.cpu().numpy(), ref_c) <= 1e-12
    assert rel(of.cpu().numpy(), ref_f) <= 1e-12


@pytest.mark.parametrize("scheme,flags", [(1, 0), (0, B.FLAG_CSR)])
def test_increments_rejected_on_least_squares_and_sparse_row_plans(scheme, flags):
    items, c, f = _batch([3] * 3, [scheme] * 3)
    plan = B.Plan(items, 7, len(c), len(f), B.PREC_SPLIT, flags)
    incr = torch.empty(plan.info["increment_elems"], dtype=torch.float32, device="cuda")
    with pytest.raises(B.AmrError):
        plan.interpolate_increments(torch.as_tensor(c).cuda(), incr)


@pytest.mark.parametrize("precision,tol_i", [(B.PREC_FP64, 1e-12), (B.PREC_SPLIT, 2e-6)])
def test_least_squares_factorised_equals_sparse_rows(precision, tol_i):
    """The same least-squares operators through the factorised kernels and
    through the sparse-row kernels (AMR_FLAG_CSR), with the one-warp-per-
    centre mapping on the factorised side."""
    items, c, f = _batch([3, 2, 3, 3, 2, 3], [1] * 6, U=31, seed=13)
    a = B.Plan(items, 31, len(c), len(f), precision)
    if precision == B.PREC_SPLIT:
        a.set_tuning(384, 112 * 1024, 256, 2, 32)
    b = B.Plan(items, 31, len(c), len(f), precision, B.FLAG_CSR)
    fa, fb = gpu_interpolate(a, c, f), gpu_interpolate(b, c, f)
    fm, cm = written_masks(items, 31, len(c), len(f))
    assert normwise_errors(items, 31, fa, fb, fm, "fine")[0] <= tol_i
    ca, cb = gpu_restrict(a, f, c), gpu_restrict(b, f, c)
    tol_r = 1e-12 if precision == B.PREC_FP64 else SPLIT_RESTRICT_TOL
    assert normwise_errors(items, 31, ca, cb, cm, "coarse")[0] <= tol_r
